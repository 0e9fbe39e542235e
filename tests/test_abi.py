"""The C ABI library builds for sm_103a, loads, and exports every entry point that
include/vcmdp.h declares (no GPU needed: nothing here calls into the device)."""
import os
import re
import subprocess

from paper_2012_12419_gb300 import build as vbuild
from paper_2012_12419_gb300 import native

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "vcmdp.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(vc_\w+)\s*\(", src, flags=re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    path = vbuild.build()
    assert os.path.exists(path)
    names = declared_functions()
    assert len(names) >= 10
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (vc_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert set(native.EXPORTS) <= set(names)
    assert set(native.exported_symbols(path)) == set(native.EXPORTS)


def test_library_targets_sm103a_only():
    path = vbuild.build()
    out = subprocess.run(["cuobjdump", "--list-elf", path], capture_output=True, text=True)
    if out.returncode != 0:
        return  # cuobjdump unavailable: nothing to check
    archs = set(re.findall(r"sm_(\d+a?)", out.stdout))
    assert archs == {"103a"}, archs


def test_binding_constants_equal_the_header():
    """Every integer #define of the header that the binding also names has the same value
    (status codes, storage forms, value types, iteration flags)."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    defs = {k: int(v) for k, v in re.findall(r"^#define\s+(VC_\w+)\s+(-?\d+)\s*$", src, flags=re.M)}
    shared = [k for k in defs if hasattr(native, k)]
    assert {"VC_OK", "VC_ITER_FP32_ONLY", "VC_ITER_SELF_LOOP", "VC_SLICED"} <= set(shared)
    for k in shared:
        assert getattr(native, k) == defs[k], k
    # the iteration flags are distinct bits
    flags = [defs[k] for k in defs if k.startswith("VC_ITER_")]
    assert all(f > 0 and f & (f - 1) == 0 for f in flags) and len(set(flags)) == len(flags)
