"""Pins of the oracle routines that the parity tests and the CPU baselines lean on, each
against facts fixed outside the oracle's code:

* the greedy heuristic (Algorithm 2 read as a policy) against a table of actions worked
  by hand (``tests/golden/greedy_policy.txt``): states where the rate order, a full host,
  the control-channel phase, an empty queue and equal rates each decide the action;
* the sampled sweep that times the oracle (``sweep_states``) against the hand-derived
  transition rows of ``tests/golden/rows_h2c2q1.txt`` (its Bellman values and its count
  of successor terms), against the closed successor count of the tiny workload, and
  against the single-state backup on every state;
* the threaded whole-state backup used at full size (``backup_all``) against the
  single-state backup, independent of how the states are split over threads.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

from test_oracle_model import H2C2Q1, _read_golden


def _read_greedy(path):
    blocks = []
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            if parts[0] == "instance":
                H, C, Q = int(parts[1]), int(parts[2]), int(parts[3])
                mu = [float(x) for x in parts[4:4 + H]]
                assert len(mu) == H
                p = dict(H=H, C=C, Q=Q, gamma=0.95, lam=1.0, mu=mu, delta=[0.125] * H, f=0.25, w_occ=1.0,
                         w_loss=-5.0, w_q=-0.1)
                blocks.append((p, []))
                continue
            vals = [int(x) for x in parts]
            H = blocks[-1][0]["H"]
            assert len(vals) == H + 3
            blocks[-1][1].append((vals[:H], vals[H], vals[H + 1], vals[H + 2]))
    return blocks


def _code(p, occ, q, ph):
    # Eq. 10's mixed-radix state code, written out here from its definition
    C, Q = p["C"], p["Q"]
    return ph + 2 * (q + (Q + 1) * sum(o * (C + 1) ** k for k, o in enumerate(occ)))


def test_greedy_policy_matches_hand_worked_actions(golden_dir):
    blocks = _read_greedy(os.path.join(golden_dir, "greedy_policy.txt"))
    assert len(blocks) == 4
    n = 0
    for p, rows in blocks:
        pi = oracle.greedy_policy(p)
        assert len(pi) == oracle.num_states(p)
        for occ, q, ph, want in rows:
            s = _code(p, occ, q, ph)
            assert pi[s] == want, (p["mu"], occ, q, ph, pi[s], want)
            n += 1
    assert n == 23


def test_greedy_policy_is_always_feasible_and_defers_only_when_it_must():
    # every state of the tiny workload: the chosen action is feasible; defer is chosen
    # exactly when no host is feasible; a placement never goes to a slower feasible host
    p = inputs.workload("tiny")
    H = p["H"]
    pi = oracle.greedy_policy(p)
    for s in range(oracle.num_states(p)):
        feas = [a for a in range(H) if oracle.feasible(p, s, a)]
        assert oracle.feasible(p, s, int(pi[s]))
        if not feas:
            assert pi[s] == H
        else:
            assert pi[s] in feas
            assert all(p["mu"][a] <= p["mu"][pi[s]] for a in feas)


def test_sweep_states_against_the_hand_derived_rows(golden_dir):
    rows = _read_golden(os.path.join(golden_dir, "rows_h2c2q1.txt"))
    S = oracle.num_states(H2C2Q1)
    g = np.random.default_rng(5)
    # dyadic values: every product and sum below is exact in FP64
    V = g.integers(-64, 64, S).astype(np.float64) / 8.0
    gamma = H2C2Q1["gamma"]
    by_state = {}
    for s, a, R, cols, probs in rows:
        by_state.setdefault(s, []).append((R, cols, probs))
    checked = 0
    for s, rs in by_state.items():
        if len(rs) != H2C2Q1["H"] + 1:
            continue  # a state whose rows are not all in the file
        checked += 1
        want = -np.inf
        terms = 0
        for R, cols, probs in rs:
            if R is None:
                continue
            want = max(want, R + gamma * sum(pr * V[c] for c, pr in zip(cols, probs)))
            terms += len(cols)
        Vn = np.full(S, np.nan)
        got_terms = oracle.sweep_states(H2C2Q1, V, Vn, s, s + 1)
        assert got_terms == terms, s
        assert Vn[s] == pytest.approx(want, rel=1e-15, abs=1e-15), s
        assert np.isnan(np.delete(Vn, s)).all()
    assert checked == 3


def test_sweep_states_counts_and_values_on_the_tiny_workload():
    p = inputs.workload("tiny")
    S = oracle.num_states(p)
    V = np.random.default_rng(2).random(S) * 80
    Vn = np.empty(S)
    # every state once: the canonical successor count, fixed independently (9,696)
    assert oracle.sweep_states(p, V, Vn, 0, S) == 9696
    for s in range(S):
        b, _, _ = oracle.backup(p, V, s)
        assert Vn[s] == pytest.approx(b, rel=1e-14)
    # strided sample: counts add up over the residues
    total = 0
    for r in range(4):
        Vs = np.full(S, np.nan)
        total += oracle.sweep_states(p, V, Vs, r, S, 4)
        assert np.all(np.isnan(Vs[(np.arange(S) % 4) != r]))
        assert np.array_equal(Vs[r::4], Vn[r::4])
    assert total == 9696


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_backup_all_equals_single_state_backups(threads):
    p = inputs.make_params(3, 2, 3, 0.9, seed=21)
    S = oracle.num_states(p)
    V = np.random.default_rng(threads).normal(10, 3, S)
    Vn, pi, gap = oracle.backup_all(p, V, threads=threads)
    for s in range(S):
        b, a, gp = oracle.backup(p, V, s)
        assert Vn[s] == b and pi[s] == a and gap[s] == gp
    pi2, gap2 = oracle.policy(p, V)
    assert np.array_equal(pi, pi2) and np.array_equal(gap, gap2)
