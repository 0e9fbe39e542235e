"""The bounds-checking build (the stand-in for a device memory checker, which this pool does
not offer): every data-derived index of the sweep kernels -- CSR and sliced columns, staged
row and record extents, ring placement, implicit successors -- is checked on the device;
a failed check raises a flag that the solve reports as an error.  A child process loads
that build (VC_DEBUG_BOUNDS=1) and runs every storage form and kernel variant to a
certified solve on instances with ragged tails; none may trip a check, and the values must
still match the oracle."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
import oracle
from paper_2012_12419_gb300 import inputs, native

L = native.load(build_if_missing=True)
assert L._name.endswith("libvcmdp_debug.so"), L._name
forms = [dict(fmt="implicit"), dict(fmt="csr_f32"), dict(fmt="csr_f32", padded=True), dict(fmt="csr_bf16"),
         dict(fmt="csr_bf16", padded=True), dict(fmt="csr_f32", direct=True), dict(fmt="csr_f32", sliced=True),
         dict(fmt="csr_bf16", padded=True, sliced=True), dict(fmt="csr_f32", sliced=True, direct=True)]
for p in (inputs.workload("tiny"), inputs.make_params(4, 4, 6, 0.95, seed=7)):
    Vs = oracle.solve(p, tol=1e-12)[0]
    for kw in forms:
        m = native.MDP.build(p, **kw)
        if kw.get("sliced"):
            m.autotune(reps=1)
        _, V64, pi, st = m.value_iterate(tol=1e-6)
        assert st["certified"] == 1, (kw, st)
        err = float(np.max(np.abs(V64.cpu().numpy() - Vs) / np.abs(Vs)))
        assert err <= 1e-6, (kw, err)
        m.close()
S, A = 5000, 9
mdp = inputs.random_csr_mdp(S, A, max_succ=12, seed=3, gamma=0.9)
args = (S, A, torch.tensor(mdp["row_ptr"], device="cuda"), torch.tensor(mdp["col"], device="cuda"),
        torch.tensor(mdp["val"].astype(np.float32), device="cuda"),
        torch.tensor(mdp["R"].astype(np.float32), device="cuda"), 0.9)
for sliced in (False, True):
    m = native.MDP.from_csr(*args)
    if sliced:
        m.slice()
    _, V64, pi, st = m.value_iterate(tol=1e-8)
    assert st["certified"] == 1, st
    m.close()
# the no-allocation sweep reports its checks through its static control block
for p in (inputs.workload("tiny"), inputs.make_params(4, 4, 6, 0.95, seed=7)):
    m = native.MDP.build(p, fmt="implicit")
    V = torch.rand(m.S, device="cuda") * 50
    ref = torch.empty_like(V)
    m.bellman32(V, ref)
    out = torch.empty_like(V)
    res = torch.zeros(1, device="cuda")
    native.bellman32_noalloc(p, V, out, None, res)
    torch.cuda.synchronize()
    assert torch.equal(out, ref) and res.item() == (out - V).abs().max().item()
    m.close()
print("debug bounds ok")
""".replace("ROOT", repr(ROOT))


def test_bounds_checking_build_runs_every_kernel_clean():
    env = dict(os.environ, VC_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "debug bounds ok" in r.stdout
