"""The ctypes mirrors of the C ABI's structures (paper_2012_12419_gb300/native.py) against
the header itself: a small C program compiled with the host compiler against
include/vcmdp.h prints every structure's size and every field's offset, and each must
equal the binding's.  A field added, removed, reordered or retyped on one side only fails
here, on the CPU, before any call could read the wrong bytes."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2012_12419_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
# binding field names that differ from the header's ("lambda" is a Python keyword)
C_NAME = {"lam": "lambda"}
STRUCTS = {
    "vc_params": native.Params,
    "vc_binary_params": native.BinaryParams,
    "vc_info": native.Info,
    "vc_stats": native.Stats,
    "vc_grad_stats": native.GradStats,
    "vc_batch_info_t": native.BatchInfo,
    "vc_batch_stats": native.BatchStats,
}


def _c_layouts(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "vcmdp.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {C_NAME.get(field, field)}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    got = {}
    for line in out.splitlines():
        name, key, val = line.split()
        got[(name, key)] = int(val)
    return got


def test_binding_structures_match_the_header(tmp_path):
    c = _c_layouts(tmp_path)
    for cname, py in STRUCTS.items():
        assert c[(cname, "size")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert c[(cname, field)] == getattr(py, field).offset, (cname, field)
