"""Pins of the oracle's value iteration, policy and policy evaluation (Algorithm 3,
Eq. 18) to facts fixed outside its code: exhaustive policy enumeration with dense
solves, closed forms, the contraction error bound, and optimality invariants."""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs


def test_one_state_closed_form():
    # One state, three actions, every action loops back: V = max_a R_a / (1 - gamma).
    gamma = 0.9
    P = np.ones((3, 1, 1))
    R = np.array([[0.5, 2.0, -1.0]])
    V = oracle.dense_value_iteration(P, R, gamma, tol=1e-13)
    assert V[0] == pytest.approx(2.0 / (1 - gamma), rel=1e-11)
    Vc, _ = oracle.vi_csr(1, 3, [0, 1, 2, 3], [0, 0, 0], [1.0, 1.0, 1.0], R[0], gamma, tol=1e-13)
    assert Vc[0] == pytest.approx(2.0 / (1 - gamma), rel=1e-11)


def test_h1_q0_closed_form():
    """H=1, C=1, Q=0: nothing can ever be placed.  From occ=0 the only reward is the
    blocked-arrival loss, so V0 = w_loss*(lam/Lam)/(1-gamma) in both phases; from occ=1
    the host empties at rate (mu+delta)/Lam, giving
    V1 = (R1 + gamma*p_out*V0) / (1 - gamma*(1-p_out)), R1 = w_occ + w_loss*(delta+lam)/Lam."""
    p = dict(H=1, C=1, Q=0, gamma=0.9, lam=0.7, mu=[0.6], delta=[0.05], f=0.4, w_occ=1.0, w_loss=-5.0, w_q=-0.1)
    Lam = 0.7 + 1 * 0.6 + 0.05 + 1.0
    gamma = 0.9
    V0 = -5.0 * (0.7 / Lam) / (1 - gamma)
    p_out = (0.6 + 0.05) / Lam
    R1 = 1.0 - 5.0 * (0.05 + 0.7) / Lam
    V1 = (R1 + gamma * p_out * V0) / (1 - gamma * (1 - p_out))
    V, _, _ = oracle.value_iteration(p, tol=1e-13)
    for s in range(oracle.num_states(p)):
        occ, q, ph = oracle.decode(p, s)
        want = V1 if occ[0] == 1 else V0
        assert V[s] == pytest.approx(want, rel=1e-11)


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 1, 1), (1, 2, 2)])
def test_generator_brute_force(shape):
    """V* equals the elementwise max over all deterministic policies of (I-gamma P_pi)^-1 R_pi."""
    H, C, Q = shape
    p = inputs.make_params(H, C, Q, 0.9, seed=100 + H * 10 + C)
    P, R = oracle.model_dense(p)
    Vb = oracle.brute_force_optimum(P, R, p["gamma"])
    Vo, _, _ = oracle.value_iteration(p, tol=1e-13)
    assert np.max(np.abs(Vo - Vb)) < 1e-10 * max(1.0, np.max(np.abs(Vb)))
    Vs, pi, gap, _ = oracle.solve(p, tol=1e-13)
    assert np.max(np.abs(Vs - Vb)) < 1e-10 * max(1.0, np.max(np.abs(Vb)))


@pytest.mark.parametrize("seed", range(6))
def test_random_dense_mdp_brute_force(seed):
    g = np.random.default_rng(seed)
    S = int(g.integers(2, 7))
    A = int(g.integers(1, 4))
    gamma = [0.5, 0.9, 0.95][seed % 3]
    P = g.random((A, S, S)) * (g.random((A, S, S)) < 0.6)
    P[:, :, 0] += 0.01
    P /= P.sum(axis=2, keepdims=True)
    R = g.uniform(-2, 2, (S, A))
    if A > 1:
        R[g.random((S, A)) < 0.25] = -np.inf
        R[:, 0] = g.uniform(-2, 2, S)
    Vb = oracle.brute_force_optimum(P, R, gamma)
    Vd = oracle.dense_value_iteration(P, R, gamma, tol=1e-13)
    assert np.max(np.abs(Vd - Vb)) < 1e-10
    # same MDP through the CSR oracle
    row_ptr, col, val, Rf = [0], [], [], []
    for s in range(S):
        for a in range(A):
            nz = np.nonzero(P[a, s])[0] if R[s, a] != -np.inf else []
            col.extend(nz.tolist() if len(nz) else [])
            val.extend(P[a, s, nz].tolist() if len(nz) else [])
            row_ptr.append(len(col))
            Rf.append(R[s, a])
    Vc, _ = oracle.vi_csr(S, A, row_ptr, col, val, Rf, gamma, tol=1e-13)
    assert np.max(np.abs(Vc - Vb)) < 1e-10


def test_q0_is_a_markov_reward_process():
    """With Q = 0 only 'defer' is feasible: VI must equal the dense solve of the chain."""
    p = inputs.make_params(2, 2, 0, 0.95, seed=21)
    S = oracle.num_states(p)
    pi = np.full(S, p["H"], np.int32)
    Vd = oracle.policy_eval_dense(p, pi)
    Vo, _, _ = oracle.value_iteration(p, tol=1e-13)
    assert np.max(np.abs(Vo - Vd)) < 1e-10 * np.max(np.abs(Vd))


def test_error_bound_and_contraction():
    """||V_k - V*|| <= gamma/(1-gamma) * ||V_k - V_{k-1}|| and residuals shrink by gamma."""
    p = inputs.workload("tiny")
    gamma = p["gamma"]
    Vstar, _, _, _ = oracle.solve(p, tol=1e-13)
    for eps in (1e-2, 1e-4, 1e-6):
        V, k, res, hist = oracle.value_iteration(p, tol=eps, record=True)
        assert res < eps
        err = np.max(np.abs(V - Vstar))
        assert err <= gamma / (1 - gamma) * res + 1e-12
        # contraction up to FP64 rounding of |V| ~ 1e2
        assert np.all(hist[1:] <= gamma * hist[:-1] + 1e-12)


def test_policy_evaluation_iter_matches_dense():
    p = inputs.workload("tiny")
    pi = oracle.greedy_policy(p)
    Vd = oracle.policy_eval_dense(p, pi)
    Vi = oracle.policy_eval_iter(p, pi, tol=1e-13)
    assert np.max(np.abs(Vi - Vd)) < 1e-10


def test_greedy_and_random_policies_never_beat_optimum():
    p = inputs.workload("tiny")
    Vstar, pistar, gap, _ = oracle.solve(p, tol=1e-13)
    Vg = oracle.policy_eval_dense(p, oracle.greedy_policy(p))
    assert np.all(Vg <= Vstar + 1e-9)
    g = np.random.default_rng(3)
    S = oracle.num_states(p)
    for _ in range(5):
        pi = np.empty(S, np.int32)
        for s in range(S):
            acts = [a for a in range(p["H"] + 1) if oracle.feasible(p, s, a)]
            pi[s] = acts[int(g.integers(len(acts)))]
        Vr = oracle.policy_eval_dense(p, pi)
        assert np.all(Vr <= Vstar + 1e-9)
    # the optimal policy's dense value satisfies the Bellman equation itself
    for s in range(0, S, 7):
        b, a, _ = oracle.backup(p, Vstar, s)
        assert b == pytest.approx(Vstar[s], abs=1e-9)
        assert a == pistar[s]


def test_policy_ties_go_to_lowest_action():
    # two identical actions: argmax must be the lower one, gap zero
    P = np.ones((2, 1, 1))
    S, A = 1, 2
    pi, gap = oracle.policy_csr(S, A, [0, 1, 2], [0, 0], [1.0, 1.0], [1.0, 1.0], 0.5, [2.0])
    assert pi[0] == 0 and gap[0] == 0.0
    pi, gap = oracle.policy_csr(S, A, [0, 1, 2], [0, 0], [1.0, 1.0], [1.0, 3.0], 0.5, [2.0])
    assert pi[0] == 1 and gap[0] == pytest.approx(2.0)
    pi, gap = oracle.policy_csr(S, A, [0, 1, 1], [0], [1.0], [1.0, -np.inf], 0.5, [2.0])
    assert pi[0] == 0 and gap[0] == np.inf


def test_tiny_workload_reference_numbers():
    """Sanity of the tiny workload's optimum: finite, inside the reward bounds / (1-gamma)."""
    p = inputs.workload("tiny")
    V, pi, gap, sweeps = oracle.solve(p, tol=1e-12)
    rmax = p["H"] * p["C"] * 1.0
    rmin = p["w_q"] * p["Q"] + p["w_loss"] * (p["C"] * sum(p["delta"]) + p["lam"]) / oracle.uniformisation(p)
    assert np.all(V <= rmax / (1 - p["gamma"]) + 1e-9)
    assert np.all(V >= rmin / (1 - p["gamma"]) - 1e-9)
    assert 100 < sweeps < 2000
