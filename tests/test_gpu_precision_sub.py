"""BF16 storage on the precision form's sub-instance (H=5 C=4 Q=15: 100,000 states, six
actions, 3,322,500 non-zero successors), where the oracle solves both matrices exactly:

* the FP32 iterate of every BF16 handle (canonical and padded rows, CSR and sliced sweeps)
  matches the oracle's fixed point of the renormalised BF16 matrix within the FP32 bound
  (contraction from the stopping residual, rounding over 1/(1-gamma) sweeps, the scaled
  rows' sum defect);
* the certified V64 of every handle matches the exact-P optimum within 1e-6 relative (the
  refinement and certificate use the exact model), and the policy equals the exact argmax
  where its gap exceeds 1e-6;
* the modelling error of BF16 storage itself -- the distance between the BF16 matrix's
  optimum and the exact optimum -- is stated: 1.65e-3 relative at most (0.081 on values
  up to 308), below the bound 2^-8 gamma/(1-gamma) relative of one BF16 rounding per entry.
"""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

from gpu_common import native_or_skip, policy_mismatches, rel_err

_cache = {}


def _references():
    if not _cache:
        p = inputs.workload("precision_sub")
        S, A = oracle.num_states(p), oracle.num_actions(p)
        rp, col, val, R = oracle.build_csr(p)
        _, eff, _ = oracle.bf16_renormalised(rp, val, len(R))
        R32 = R.astype(np.float32).astype(np.float64)
        Vb, _ = oracle.vi_csr(S, A, rp, col, eff, R32, p["gamma"], tol=1e-10)
        Vs, _ = oracle.vi_csr(S, A, rp, col, val, R, p["gamma"], tol=1e-10)
        pis, gaps = oracle.policy_csr(S, A, rp, col, val, R, p["gamma"], Vs)
        _cache.update(p=p, Vb=Vb, Vs=Vs, pis=pis, gaps=gaps)
    return _cache


def test_bf16_modelling_error_on_the_sub_instance():
    ref = _references()
    p = ref["p"]
    err = rel_err(ref["Vb"], ref["Vs"])
    assert err <= 1.7e-3
    assert err <= 2.0**-8 * p["gamma"] / (1 - p["gamma"])


@pytest.mark.gpu
@pytest.mark.parametrize("padded,sliced", [(False, False), (True, False), (False, True), (True, True)])
def test_bf16_handles_on_the_sub_instance(padded, sliced):
    native = native_or_skip()
    ref = _references()
    p = ref["p"]
    m = native.MDP.build(p, fmt="csr_bf16", padded=padded, sliced=sliced)
    V, V64, pi, st = m.value_iterate(tol=1e-6)
    assert st["certified"] == 1
    V32 = V.cpu().numpy().astype(np.float64)
    vmax = float(np.max(np.abs(ref["Vb"])))
    g = p["gamma"]
    ulp = float(np.spacing(np.float32(vmax)))
    bound = g / (1 - g) * st["residual"] + 2 * ulp / (1 - g) + g * 2.0**-24 * vmax / (1 - g)
    assert np.max(np.abs(V32 - ref["Vb"])) <= bound
    assert rel_err(V64.cpu().numpy(), ref["Vs"]) <= 1e-6
    assert policy_mismatches(pi.cpu().numpy(), ref["pis"], ref["gaps"])[0] == 0
    m.close()
