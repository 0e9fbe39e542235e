"""Pins of the oracle's binary-action model (the paper's A = {-1, 1}, Section V-B..V-E, with
the transition law read as one uniformised event per step), each against a fact fixed
outside the oracle's code:

* hand-derived rows of a dyadic instance (``tests/golden/rows_binary_h2c2j2.txt``):
  columns, merging, ordering, probabilities, both rewards, feasibility;
* the state code's definition, rows are distributions with at most 2H + 1 + HJ entries;
* brute force: the optimum equals the best of every deterministic policy's dense solve;
* the threaded whole-state backup against a dense backup of the tiny instance;
* a closed form: under "always -1" (every task to the paid cloud) the empty system stays
  empty, and its values are W = gamma q rbar / (1 - gamma) with no request pending and
  r(i, n) + W with a request (q = lambda / Lam the probability of a request, rbar the mean
  immediate reward of a request sent to the paid cloud).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

DYADIC = dict(H=2, C=2, J=2, gamma=0.95, lam=1.0, mu=[0.5, 0.25], delta=[0.25, 0.25], beta_vc=1.0, beta_tc=1.2,
              gamma_vc=1.0)


def _read(path):
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            head, _, tail = line.partition("|")
            parts = head.split()
            s, a = int(parts[0]), int(parts[1])
            if parts[2] == "infeasible":
                rows.append((s, a, None, None, None))
                continue
            cols, probs = [], []
            for tok in tail.split():
                c, pr = tok.split(":")
                cols.append(int(c))
                probs.append(float(pr))
            rows.append((s, a, float(parts[2]), cols, probs))
    return rows


def test_hand_derived_rows(golden_dir):
    rows = _read(os.path.join(golden_dir, "rows_binary_h2c2j2.txt"))
    assert len(rows) == 10
    assert oracle.bin_num_states(DYADIC) == 45
    assert oracle.bin_uniformisation(DYADIC) == 4.0
    for s, a, R, cols, probs in rows:
        got = oracle.bin_transitions(DYADIC, s, a)
        if R is None:
            assert got is None, (s, a)
            continue
        gc, gp, gR = got
        assert gc.tolist() == cols, (s, a)
        assert gp.tolist() == probs, (s, a)  # dyadic: exact
        assert gR == pytest.approx(R, abs=1e-14), (s, a)


def _code(p, u, e):
    E = 1 + p["H"] * p["J"]
    return e + E * sum(x * (p["C"] + 1) ** k for k, x in enumerate(u))


@pytest.mark.parametrize("name", ["binary_tiny", "binary_mid"])
def test_rows_are_distributions_and_the_state_code(name):
    p = inputs.binary_workload(name)
    H, C, J = p["H"], p["C"], p["J"]
    S = oracle.bin_num_states(p)
    assert S == inputs.binary_num_states(H, C, J) == (1 + H * J) * (C + 1) ** H
    rp, col, val, R = oracle.bin_build_csr(p)
    assert rp[-1] == len(col)
    n = np.diff(rp)
    assert n.max() <= 2 * H + 1 + H * J
    for r in range(2 * S):
        if not np.isfinite(R[r]):
            assert n[r] == 0
            continue
        c = col[rp[r]:rp[r + 1]]
        v = val[rp[r]:rp[r + 1]]
        assert np.all(np.diff(c) > 0) and np.all(v > 0)
        assert abs(v.sum() - 1.0) < 1e-14
    # every state with no request has exactly the no-op; -1 is always feasible
    E = 1 + H * J
    for s in range(S):
        e = s % E
        assert np.isfinite(R[2 * s])
        if e == 0:
            assert not np.isfinite(R[2 * s + 1]) and R[2 * s] == 0.0
    # feasibility of +1 by the digits, written out from the definition
    g = np.random.default_rng(1)
    for _ in range(200):
        u = [int(x) for x in g.integers(0, C + 1, H)]
        i, m = int(g.integers(H)), int(g.integers(1, J + 1))
        s = _code(p, u, 1 + i * J + m - 1)
        fits = u[i] + m <= C
        assert np.isfinite(R[2 * s + 1]) == fits
        if fits:
            assert R[2 * s + 1] == pytest.approx(p["beta_vc"] * m - p["gamma_vc"] * (C - u[i] - m), abs=1e-14)
        assert R[2 * s] == pytest.approx(-p["beta_tc"] * m - p["gamma_vc"] * (C - u[i]), abs=1e-14)


def _dense(p):
    S = oracle.bin_num_states(p)
    P = np.zeros((2, S, S))
    R = np.full((S, 2), -np.inf)
    for s in range(S):
        for a in range(2):
            row = oracle.bin_transitions(p, s, a)
            if row is None:
                continue
            c, v, r = row
            P[a, s, c] = v
            R[s, a] = r
    return P, R


@pytest.mark.parametrize("H,C,J,seed", [(1, 2, 1, 1), (2, 1, 1, 2), (1, 3, 2, 3)])
def test_optimum_by_brute_force(H, C, J, seed):
    p = inputs.binary_params(H, C, J, 0.9, seed)
    P, R = _dense(p)
    best = oracle.brute_force_optimum(P, R, p["gamma"])
    V, pi, gap, _ = oracle.bin_solve(p, tol=1e-13)
    assert np.max(np.abs(V - best)) < 1e-9


def test_always_paid_cloud_closed_form():
    p = inputs.binary_params(3, 3, 2, 0.95, 9)
    H, C, J, gamma = p["H"], p["C"], p["J"], p["gamma"]
    S = oracle.bin_num_states(p)
    P, R = _dense(p)
    Pp = P[0]
    Rp = R[:, 0]
    V = np.linalg.solve(np.eye(S) - gamma * Pp, Rp)
    q = p["lam"] / oracle.bin_uniformisation(p)
    rbar = -p["beta_tc"] * (J + 1) / 2 - p["gamma_vc"] * C
    W = gamma * q * rbar / (1 - gamma)
    assert V[0] == pytest.approx(W, rel=1e-12)
    for i in range(H):
        for m in range(1, J + 1):
            e = 1 + i * J + m - 1
            assert V[e] == pytest.approx(-p["beta_tc"] * m - p["gamma_vc"] * C + W, rel=1e-12)


@pytest.mark.parametrize("threads", [1, 4])
def test_backup_all_equals_the_dense_backup(threads):
    p = inputs.binary_workload("binary_tiny")
    P, R = _dense(p)
    S = P.shape[1]
    V = np.random.default_rng(threads).normal(0, 5, S)
    Q = np.where(np.isfinite(R), R + p["gamma"] * np.einsum("ast,t->sa", P, V), -np.inf)
    Vn, pi, gap = oracle.bin_backup_all(p, V, threads=threads)
    assert np.allclose(Vn, Q.max(axis=1), rtol=1e-14, atol=1e-13)
    assert np.array_equal(pi, np.argmax(Q, axis=1))
    two = np.isfinite(Q).all(axis=1)
    assert np.allclose(gap[two], np.abs(Q[two, 0] - Q[two, 1]), rtol=1e-12, atol=1e-12)
    assert np.all(np.isinf(gap[~two]))
