"""The refinement's correction solve by BiCGSTAB against the fixed-point sweeps it replaces
and against the oracle.

* On the implicit model (a gamma = 0.95 and a gamma = 0.99 instance), on the stored rows of a
  user CSR (no model: the products read the rows of pi), and on BF16 storage (the products
  use the exact model), both correction solvers end certified, with V64 within 1e-6
  relative of the oracle's optimum and the oracle's policy wherever its Q-gap exceeds 1e-6.
* On the gamma = 0.99 instance BiCGSTAB spends fewer products by P_pi than the sweeps.
* The solve is deterministic: two runs give bitwise equal V64 and the same product count.
* vc_evaluate_policy (BiCGSTAB inside) evaluates a fixed policy of a user CSR to the
  oracle's value iteration of the single-action MDP that keeps only the policy's rows.
* The batched refinement (BiCGSTAB for every instance in one graph) against its fixed-point
  sweeps and the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

from gpu_common import native_or_skip, policy_mismatches, rel_err

pytestmark = pytest.mark.gpu

MODEL_CASES = [
    ("g95", inputs.make_params(4, 4, 6, 0.95, seed=7), dict(fmt="implicit")),
    ("g99", inputs.make_params(3, 4, 8, 0.99, seed=5), dict(fmt="implicit")),
    ("g99_csr", inputs.make_params(3, 4, 8, 0.99, seed=5), dict(fmt="csr_f32", sliced=True)),
    ("bf16", inputs.make_params(4, 4, 6, 0.95, seed=7), dict(fmt="csr_bf16", padded=True)),
]
_ref = {}


def _oracle(name, p):
    if name not in _ref:
        _ref[name] = oracle.solve(p, tol=1e-12)
    return _ref[name]


@pytest.mark.parametrize("name,p,kw", MODEL_CASES, ids=[c[0] for c in MODEL_CASES])
def test_bicgstab_and_sweeps_agree_with_the_oracle(name, p, kw):
    native = native_or_skip()
    Vs, pis, gaps, _ = _oracle(name, p)
    m = native.MDP.build(p, **kw)
    out = {}
    for plain in (False, True):
        _, V64, pi, st = m.value_iterate(tol=1e-6, plain_correction=plain)
        assert st["certified"] == 1, (plain, st)
        assert rel_err(V64.cpu().numpy(), Vs) <= 1e-6
        assert policy_mismatches(pi.cpu().numpy(), pis, gaps)[0] == 0
        out[plain] = (V64.cpu().numpy(), st)
    # the two certified results are both within gamma/(1-gamma) tol of V*
    g = p["gamma"]
    assert np.max(np.abs(out[False][0] - out[True][0])) <= 2 * g / (1 - g) * 1e-6
    if name == "g99":
        assert out[False][1]["eval_sweeps"] < out[True][1]["eval_sweeps"]
    m.close()


def test_bicgstab_solve_is_deterministic():
    native = native_or_skip()
    import torch

    p = MODEL_CASES[1][1]
    m = native.MDP.build(p, fmt="implicit")
    _, Va, pa, sa = m.value_iterate(tol=1e-6)
    _, Vb, pb, sb = m.value_iterate(tol=1e-6)
    assert torch.equal(Va, Vb) and torch.equal(pa, pb)
    assert sa["eval_sweeps"] == sb["eval_sweeps"] and sa["eval_sweeps"] > 0
    m.close()


def test_user_csr_stored_rows_and_policy_evaluation():
    native = native_or_skip()
    import torch

    S, A, gamma = 3000, 5, 0.97
    mdp = inputs.random_csr_mdp(S, A, max_succ=9, seed=11, gamma=gamma)
    rp, col, val, R = mdp["row_ptr"], mdp["col"], mdp["val"], mdp["R"]
    dev = "cuda"
    m = native.MDP.from_csr(S, A, torch.tensor(rp, device=dev), torch.tensor(col, device=dev),
                            torch.tensor(val.astype(np.float32), device=dev),
                            torch.tensor(R.astype(np.float32), device=dev), gamma)
    # the device holds FP32 probabilities and rewards: the oracle solves that matrix
    val32 = val.astype(np.float32).astype(np.float64)
    R32 = R.astype(np.float32).astype(np.float64)
    Vs, _ = oracle.vi_csr(S, A, rp, col, val32, R32, gamma, tol=1e-12)
    pis, gaps = oracle.policy_csr(S, A, rp, col, val32, R32, gamma, Vs)
    for plain in (False, True):
        _, V64, pi, st = m.value_iterate(tol=1e-6, plain_correction=plain)
        assert st["certified"] == 1
        assert rel_err(V64.cpu().numpy(), Vs) <= 1e-6
        assert policy_mismatches(pi.cpu().numpy(), pis, gaps)[0] == 0
    # a fixed feasible policy (the lowest feasible action but one where possible)
    feas = np.isfinite(R.reshape(S, A))
    pol = np.array([np.flatnonzero(f)[min(1, f.sum() - 1)] for f in feas], np.int32)
    Rpol = np.full(S * A, -np.inf)
    rows = np.arange(S) * A + pol
    Rpol[rows] = R32[rows]
    Vpol, _ = oracle.vi_csr(S, A, rp, col, val32, Rpol, gamma, tol=1e-13)
    Vp, n = m.evaluate_policy(torch.tensor(pol, device=dev), tol=1e-10)
    assert n > 0
    assert np.max(np.abs(Vp.cpu().numpy() - Vpol) / np.maximum(np.abs(Vpol), 1.0)) <= 1e-9
    m.close()


def test_batched_bicgstab_against_sweeps_and_oracle():
    """Batched refinement: BiCGSTAB for every instance (one graph) against the fixed-point
    sweeps, on small uneven instances with gamma in {0.9, 0.95, 0.99}: both certified in
    accuracy mode and within tol/2 of the oracle's optimum; BiCGSTAB spends fewer products
    on the gamma = 0.99 instances; two BiCGSTAB runs are bitwise equal."""
    native = native_or_skip()
    ps = [p for p in inputs.batch_params(512, seed=2) if inputs.num_states(p["H"], p["C"], p["Q"]) <= 4000][:18]
    assert {p["gamma"] for p in ps} == {0.9, 0.95, 0.99}
    b = native.Batch(ps)
    res = {}
    for plain in (False, True):
        V, V64, pi, stats, rc = b.value_iterate(tol=1e-6, accurate=True, plain_correction=plain)
        assert rc == native.VC_OK
        assert all(s["certified"] == 1 for s in stats)
        res[plain] = (V64.cpu().numpy(), pi.cpu().numpy(), stats)
    off = b.offsets
    prods = {False: 0, True: 0}
    for i, p in enumerate(ps):
        sl = slice(off[i], off[i + 1])
        Vs, pis, gaps, _ = oracle.solve(p, tol=1e-12)
        for plain in (False, True):
            V64, pi, stats = res[plain]
            assert np.max(np.abs(V64[sl] - Vs)) <= 5e-7 + 1e-9
            assert policy_mismatches(pi[sl], pis, gaps)[0] == 0
            if p["gamma"] == 0.99:
                prods[plain] += stats[i]["correction_sweeps"]
    assert prods[False] < prods[True]
    _, V64b, pib, _, _ = b.value_iterate(tol=1e-6, accurate=True)
    assert np.array_equal(V64b.cpu().numpy(), res[False][0]) and np.array_equal(pib.cpu().numpy(), res[False][1])
    b.close()


def test_product_budget_and_fallback_path():
    """A product budget too small for BiCGSTAB sends the correction to the fixed-point
    fallback and then reports VC_ERR_NOT_CONVERGED; the same call with a large budget
    evaluates the policy to the oracle's values (the handle stays usable)."""
    native = native_or_skip()
    p = inputs.make_params(3, 4, 8, 0.99, seed=5)
    m = native.MDP.build(p, fmt="implicit")
    pi = m.greedy_policy()
    with pytest.raises(native.VcError):
        m.evaluate_policy(pi, tol=1e-10, max_sweeps=10)
    Vg, n = m.evaluate_policy(pi, tol=1e-10)
    Vgo = oracle.policy_eval_iter(p, pi.cpu().numpy(), tol=1e-13)
    assert n > 0
    assert np.max(np.abs(Vg.cpu().numpy() - Vgo) / np.maximum(np.abs(Vgo), 1.0)) <= 1e-9
    m.close()
