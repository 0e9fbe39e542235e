"""Pins of the oracle's gradient pieces and bfloat16 rounding.

* analytic transition derivatives vs central finite differences of the rows themselves;
* the dense-solve adjoint gradient vs central finite differences of J = rho . V*
  (valid where the optimal policy does not flip within +-h) and vs the Euler identity
  J = sum_j w_j dJ/dw_j (V* is positively 1-homogeneous in the reward weights);
* bfloat16 round-to-nearest-even vs its definition (nearest representable value,
  ties to the even mantissa) on hand-picked and random inputs.
"""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs


def _rho_empty_hosts(p):
    S = oracle.num_states(p)
    rho = np.zeros(S)
    for s in range(S):
        occ, _, _ = oracle.decode(p, s)
        if all(o == 0 for o in occ):
            rho[s] = 1.0
    return rho / rho.sum()


def test_transition_derivatives_match_finite_differences():
    p = inputs.make_params(3, 2, 2, 0.95, seed=31)
    theta = oracle.theta_vector(p)
    h = 1e-6
    g = np.random.default_rng(0)
    S = oracle.num_states(p)
    checked = 0
    for s in g.choice(S, 40, replace=False):
        for a in range(p["H"] + 1):
            got = oracle.transition_grads(p, int(s), a)
            if got is None:
                continue
            cols, dP, dR = got
            for i in range(len(theta)):
                tp, tm = theta.copy(), theta.copy()
                tp[i] += h
                tm[i] -= h
                rp = oracle.transitions(oracle.with_theta(p, tp), int(s), a)
                rm = oracle.transitions(oracle.with_theta(p, tm), int(s), a)
                assert rp[0].tolist() == cols.tolist() == rm[0].tolist()
                fd_p = (rp[1] - rm[1]) / (2 * h)
                fd_r = (rp[2] - rm[2]) / (2 * h)
                assert np.allclose(dP[:, i], fd_p, atol=1e-8, rtol=1e-6), (s, a, i)
                assert dR[i] == pytest.approx(fd_r, abs=1e-7, rel=1e-6), (s, a, i)
            checked += 1
    assert checked > 40


def _J(p, rho):
    V, _, _, _ = oracle.solve(p, tol=1e-12)
    return float(rho @ V)


def test_dense_adjoint_matches_finite_differences_and_euler():
    p = inputs.workload("tiny")
    rho = _rho_empty_hosts(p)
    assert int(np.count_nonzero(rho)) == 2 * (p["Q"] + 1)
    V, pi, gap, _ = oracle.solve(p, tol=1e-12)
    J = float(rho @ V)
    g = oracle.grad_dense(p, V, pi, rho)
    theta = oracle.theta_vector(p)
    h = 1e-4
    names = oracle.theta_names(p["H"])
    for i in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        pp, pm = oracle.with_theta(p, tp), oracle.with_theta(p, tm)
        Vp, pip, _, _ = oracle.solve(pp, tol=1e-12)
        Vm, pim, _, _ = oracle.solve(pm, tol=1e-12)
        if not (np.array_equal(pip, pi) and np.array_equal(pim, pi)):
            continue  # the policy flips inside +-h: the derivative is one-sided there
        fd = (rho @ Vp - rho @ Vm) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-6), names[i]
    # Euler identity over the reward weights (exact for a fixed optimal policy)
    H = p["H"]
    w = np.array([p["w_occ"], p["w_loss"], p["w_q"]])
    assert J == pytest.approx(float(w @ g[2 * H + 2:2 * H + 5]), rel=1e-9)


def test_contraction_and_adjoint_apply_match_dense_forms():
    """The any-size C loops used at full scale agree with the dense forms pinned above."""
    p = inputs.workload("tiny")
    rho = _rho_empty_hosts(p)
    V, pi, _, _ = oracle.solve(p, tol=1e-12)
    P, R = oracle.policy_matrices(p, pi)
    lam = np.linalg.solve((np.eye(len(R)) - p["gamma"] * P).T, rho)
    assert np.max(np.abs(oracle.adjoint_apply(p, pi, lam) - P.T @ lam)) < 1e-13
    g = oracle.grad_contract(p, V, pi, lam)
    g_dense = oracle.grad_dense(p, V, pi, rho)
    assert np.max(np.abs(g - g_dense)) < 1e-10 * np.max(np.abs(g_dense))


def test_bf16_round_to_nearest_even_cases():
    one = 0x3F80
    assert oracle.bf16_rne(1.0) == one
    assert oracle.bf16_rne(1.0 + 2.0**-8) == one            # halfway, even stays
    assert oracle.bf16_rne(1.0 + 3 * 2.0**-8) == one + 2    # halfway, rounds up to even
    assert oracle.bf16_rne(1.0 + 2.0**-8 + 2.0**-40) == one + 1  # just above halfway
    assert oracle.bf16_rne(1.0 + 2.0**-8 - 2.0**-40) == one      # just below halfway
    assert oracle.bf16_rne(0.5) == 0x3F00
    assert oracle.bf16_rne(2.0 - 2.0**-9) == 0x4000          # rounds up into the next binade
    assert oracle.bf16_to_double(0x3F81) == 1.0 + 2.0**-7


def test_bf16_is_nearest_representable():
    g = np.random.default_rng(5)
    xs = np.concatenate([g.random(2000), g.random(500) * 1e-3, g.random(200) * 1e-30])
    bits = oracle.bf16_round_array(xs)
    for x, b in zip(xs, bits):
        v = oracle.bf16_to_double(int(b))
        lo = oracle.bf16_to_double(int(b) - 1) if b > 0 else -np.inf
        hi = oracle.bf16_to_double(int(b) + 1)
        assert abs(x - v) <= abs(x - lo) and abs(x - v) <= abs(x - hi)
        if abs(x - v) == abs(x - hi) or abs(x - v) == abs(x - lo):
            assert int(b) % 2 == 0
        assert oracle.bf16_rne(float(x)) == int(b)


def test_bf16_renormalised_rows_sum_to_one():
    p = inputs.workload("tiny")
    row_ptr, col, val, R = oracle.build_csr(p)
    bits, eff, scale = oracle.bf16_renormalised(row_ptr, val, len(R))
    for r in range(len(R)):
        lo, hi = row_ptr[r], row_ptr[r + 1]
        if hi > lo:
            assert abs(eff[lo:hi].sum() - 1.0) < 2e-7  # FP32 scale rounding
            # bf16 unit roundoff is 2^-8 per entry; renormalising moves each entry by at
            # most the row's total rounding (another 2^-8), so 2^-7 relative bounds it
            assert np.all(np.abs(eff[lo:hi] - val[lo:hi]) <= 2.0**-7 * val[lo:hi] + 2e-7)
