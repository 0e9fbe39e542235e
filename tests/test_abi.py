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
