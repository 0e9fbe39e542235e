"""Pins of the oracle's value iteration with each action's self-transition solved exactly
(Puterman 1994, Sec. 6.3.3; Algorithm 4's in-block iteration for a block of one state,
iterated to its limit):  Qs(s,a) = (R + gamma sum_{s' != s} P V) / (1 - gamma P(s|s,a)).

* a one-state MDP reaches the closed form max_a R_a / (1 - gamma) in one sweep;
* a two-state chain worked out by hand reaches V* exactly in two sweeps;
* without self-transitions the sweeps are those of plain value iteration, bit for bit;
* the fixed point is V* (brute-force policy enumeration on dense random MDPs, the pinned
  optimum of the tiny placement model) and each sweep contracts the error by at most
  max_{s,a} gamma (1 - p_ss) / (1 - gamma p_ss);
* the model form and the CSR form of the oracle agree, with fewer sweeps than Eq. 18's.
"""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs


def _dense_to_csr(P, R):
    A, S, _ = P.shape
    rp, col, val, Rr = [0], [], [], []
    for s in range(S):
        for a in range(A):
            if R[s, a] != -np.inf:
                nz = np.flatnonzero(P[a, s])
                col += nz.tolist()
                val += P[a, s, nz].tolist()
            rp.append(len(col))
            Rr.append(R[s, a])
    return (np.array(rp, np.int64), np.array(col, np.int32), np.array(val, np.float64), np.array(Rr, np.float64))


def _random_dense(S, A, seed, self_weight):
    rng = np.random.default_rng(seed)
    P = rng.random((A, S, S)) * (rng.random((A, S, S)) < 0.5)
    for a in range(A):
        P[a] += np.diag(self_weight * rng.random(S) * S)
        P[a] /= P[a].sum(1, keepdims=True)
    R = rng.normal(size=(S, A))
    R[rng.random((S, A)) < 0.25] = -np.inf
    R[:, 0] = rng.normal(size=S)  # every state keeps a feasible action
    return P, R


def test_one_state_reaches_the_closed_form_in_one_sweep():
    g = 0.95
    Rr = np.array([0.3, 1.7, -2.0])
    rp = np.array([0, 1, 2, 3], np.int64)
    col = np.zeros(3, np.int32)
    val = np.ones(3)
    V, n = oracle.vi_csr_self_loop(1, 3, rp, col, val, Rr, g, tol=1e-300, max_sweeps=1, strict=False)
    assert n == 1 and V[0] == pytest.approx(1.7 / (1 - g), rel=1e-15)
    # Eq. 18's backup needs ~log(tol)/log(gamma) sweeps for the same point
    V2, n2 = oracle.vi_csr(1, 3, rp, col, val, Rr, g, tol=1e-9)
    assert n2 > 400 and V2[0] == pytest.approx(1.7 / (1 - g), abs=1e-7)


def test_two_state_chain_by_hand():
    # state 0: stay w.p. 1/2, else move to the absorbing state 1; R = (1, 2), gamma = 0.9.
    # V*(1) = 2 / 0.1 = 20, V*(0) = (1 + 0.9 * 0.5 * 20) / (1 - 0.45) = 10 / 0.55.
    # Sweep 1 from 0: V(1) = 20 exactly, V(0) = 1 / 0.55; sweep 2: V(0) = 10 / 0.55.
    rp = np.array([0, 2, 3], np.int64)
    col = np.array([0, 1, 1], np.int32)
    val = np.array([0.5, 0.5, 1.0])
    Rr = np.array([1.0, 2.0])
    V1, _ = oracle.vi_csr_self_loop(2, 1, rp, col, val, Rr, 0.9, tol=1e-300, max_sweeps=1, strict=False)
    assert V1 == pytest.approx([1 / 0.55, 20.0], rel=1e-15)
    V2, _ = oracle.vi_csr_self_loop(2, 1, rp, col, val, Rr, 0.9, tol=1e-300, max_sweeps=2, strict=False)
    assert V2 == pytest.approx([10 / 0.55, 20.0], rel=1e-15)


def test_without_self_transitions_the_sweeps_are_plain_value_iteration():
    rng = np.random.default_rng(3)
    S, A = 40, 3
    P = rng.random((A, S, S)) * (rng.random((A, S, S)) < 0.3)
    for a in range(A):
        np.fill_diagonal(P[a], 0.0)
        P[a, np.arange(S), (np.arange(S) + 1) % S] += 0.1
        P[a] /= P[a].sum(1, keepdims=True)
    R = rng.normal(size=(S, A))
    rp, col, val, Rr = _dense_to_csr(P, R)
    for k in (1, 2, 7):
        Va, _ = oracle.vi_csr(S, A, rp, col, val, Rr, 0.93, tol=1e-300, max_sweeps=k, strict=False)
        Vb, _ = oracle.vi_csr_self_loop(S, A, rp, col, val, Rr, 0.93, tol=1e-300, max_sweeps=k, strict=False)
        assert np.array_equal(Va, Vb)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fixed_point_is_the_brute_force_optimum(seed):
    S, A, g = 6, 3, 0.9
    P, R = _random_dense(S, A, seed, self_weight=1.0)
    Vbf = oracle.brute_force_optimum(P, R, g)
    rp, col, val, Rr = _dense_to_csr(P, R)
    V, _ = oracle.vi_csr_self_loop(S, A, rp, col, val, Rr, g, tol=1e-14)
    assert np.max(np.abs(V - Vbf)) <= 1e-11 * np.max(np.abs(Vbf))


def test_contraction_bound_per_sweep():
    S, A, g = 8, 3, 0.95
    P, R = _random_dense(S, A, 5, self_weight=2.0)
    Vbf = oracle.brute_force_optimum(P, R, g)
    rp, col, val, Rr = _dense_to_csr(P, R)
    pss = np.array([P[a, s, s] for s in range(S) for a in range(A) if R[s, a] != -np.inf])
    kappa = np.max(g * (1 - pss) / (1 - g * pss))
    assert kappa < g
    V = np.zeros(S)
    err = np.max(np.abs(V - Vbf))
    for _ in range(30):
        V, _ = oracle.vi_csr_self_loop(S, A, rp, col, val, Rr, g, tol=1e-300, max_sweeps=1, V0=V, strict=False)
        e2 = np.max(np.abs(V - Vbf))
        assert e2 <= kappa * err * (1 + 1e-12) + 1e-12
        err = e2


def test_model_form_reaches_the_pinned_optimum_in_fewer_sweeps():
    p = inputs.make_params(3, 3, 4, 0.95, seed=0)
    Vstar = oracle.solve(p, tol=1e-13)[0]
    V, n, _ = oracle.value_iteration_self_loop(p, tol=1e-12)
    assert np.max(np.abs(V - Vstar)) <= 1e-9
    # the plain backup's residual at that point is at the tolerance's scale
    Vn = np.array([oracle.backup(p, V, s)[0] for s in range(len(V))])
    assert np.max(np.abs(Vn - V)) <= 1e-10
    # CSR form of the same instance: the same iterates, bit for bit
    S, A = oracle.num_states(p), oracle.num_actions(p)
    rp, col, val, Rr = oracle.build_csr(p)
    for k in (1, 5, 40):
        Va, _, _ = oracle.value_iteration_self_loop(p, tol=1e-300, max_sweeps=k, strict=False)
        Vb, _ = oracle.vi_csr_self_loop(S, A, rp, col, val, Rr, p["gamma"], tol=1e-300, max_sweeps=k, strict=False)
        assert np.array_equal(Va, Vb)
    _, n_plain, _ = oracle.value_iteration(p, tol=1e-12)
    assert n < n_plain


def _random_csr_with_self_loops(S, A, seed):
    rng = np.random.default_rng(seed)
    P = rng.random((A, S, S)) * (rng.random((A, S, S)) < 0.2)
    for a in range(A):
        P[a] += np.diag(rng.random(S))
        P[a, np.arange(S), (np.arange(S) + 1) % S] += 0.05
        P[a] /= P[a].sum(1, keepdims=True)
    R = rng.normal(size=(S, A))
    R[rng.random((S, A)) < 0.2] = -np.inf
    R[:, 0] = rng.normal(size=S)
    return P, R


def test_block_iteration_reduces_to_the_self_transition_sweeps():
    """passes = 1, or blocks of one state, give the sweeps of vi_csr_self_loop bit for bit;
    one block of every state with p passes is p of those sweeps."""
    S, A, g = 50, 3, 0.93
    P, R = _random_csr_with_self_loops(S, A, 4)
    rp, col, val, Rr = _dense_to_csr(P, R)
    V0 = np.random.default_rng(1).normal(size=S)
    kw = dict(tol=1e-300, V0=V0, strict=False)
    for k in (1, 4):
        ref, _ = oracle.vi_csr_self_loop(S, A, rp, col, val, Rr, g, max_sweeps=k, **kw)
        a, _ = oracle.block_vi_csr_self_loop(S, A, rp, col, val, Rr, g, 16, 1, max_sweeps=k, **kw)
        b, _ = oracle.block_vi_csr_self_loop(S, A, rp, col, val, Rr, g, 1, 3, max_sweeps=k, **kw)
        assert np.array_equal(a, ref) and np.array_equal(b, ref)
    for p in (2, 5):
        ref, _ = oracle.vi_csr_self_loop(S, A, rp, col, val, Rr, g, max_sweeps=p, **kw)
        c, _ = oracle.block_vi_csr_self_loop(S, A, rp, col, val, Rr, g, S, p, max_sweeps=1, **kw)
        assert np.array_equal(c, ref)


@pytest.mark.parametrize("seed", [0, 1])
def test_block_iteration_reaches_the_brute_force_optimum(seed):
    S, A, g = 6, 3, 0.9
    P, R = _random_dense(S, A, seed, self_weight=1.0)
    Vbf = oracle.brute_force_optimum(P, R, g)
    rp, col, val, Rr = _dense_to_csr(P, R)
    V, _ = oracle.block_vi_csr_self_loop(S, A, rp, col, val, Rr, g, 3, 4, tol=1e-14)
    assert np.max(np.abs(V - Vbf)) <= 1e-11 * np.max(np.abs(Vbf))


def test_block_iteration_on_the_model_needs_fewer_global_sweeps():
    p = inputs.make_params(3, 3, 4, 0.95, seed=0)
    S, A = oracle.num_states(p), oracle.num_actions(p)
    rp, col, val, Rr = oracle.build_csr(p)
    Vstar = oracle.solve(p, tol=1e-13)[0]
    _, n1 = oracle.vi_csr_self_loop(S, A, rp, col, val, Rr, p["gamma"], tol=1e-10)
    V, n4 = oracle.block_vi_csr_self_loop(S, A, rp, col, val, Rr, p["gamma"], 32, 4, tol=1e-10)
    assert n4 < n1
    assert np.max(np.abs(V - Vstar)) <= 1e-7
