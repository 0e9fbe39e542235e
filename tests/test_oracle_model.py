"""Pins of the oracle's model (successor enumeration, rewards, CSR form) to facts fixed
outside its code: hand-derived rows, probability axioms, the phase chain's stationary
law, closed-form counts and the state code's definition (Section V, Eq. 10-16 readings)."""
import os

import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

H2C2Q1 = dict(H=2, C=2, Q=1, gamma=0.95, lam=1.0, mu=[0.5, 0.375], delta=[0.125, 0.125], f=0.25,
              w_occ=1.0, w_loss=-5.0, w_q=-0.1)


def _read_golden(path):
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
            R = float(parts[2])
            cols, probs = [], []
            for tok in tail.split():
                c, p = tok.split(":")
                cols.append(int(c))
                probs.append(float(p))
            rows.append((s, a, R, cols, probs))
    return rows


def test_hand_derived_rows(golden_dir):
    rows = _read_golden(os.path.join(golden_dir, "rows_h2c2q1.txt"))
    assert len(rows) >= 8
    assert oracle.uniformisation(H2C2Q1) == 4.0
    for s, a, R, cols, probs in rows:
        got = oracle.transitions(H2C2Q1, s, a)
        if R is None:
            assert got is None, (s, a)
            assert not oracle.feasible(H2C2Q1, s, a)
            continue
        gc, gp, gR = got
        assert gc.tolist() == cols, (s, a)
        # dyadic instance: exact equality
        assert gp.tolist() == probs, (s, a)
        assert gR == pytest.approx(R, abs=1e-15), (s, a)


def test_state_code_definition():
    p = inputs.workload("tiny")
    H, C, Q = p["H"], p["C"], p["Q"]
    assert oracle.num_states(p) == 2 * (Q + 1) * (C + 1) ** H == 640
    seen = set()
    for s in range(oracle.num_states(p)):
        occ, q, ph = oracle.decode(p, s)
        expect = ph + 2 * (q + (Q + 1) * sum(o * (C + 1) ** k for k, o in enumerate(occ)))
        assert expect == s
        assert oracle.encode(p, occ, q, ph) == s
        seen.add((tuple(occ), q, ph))
    assert len(seen) == 640


def _small_instances():
    out = [inputs.workload("tiny"), H2C2Q1]
    out.append(inputs.make_params(2, 3, 2, 0.9, seed=11))
    out.append(inputs.make_params(1, 2, 3, 0.99, seed=12))
    return out


@pytest.mark.parametrize("idx", range(4))
def test_rows_are_distributions_with_bounded_width(idx):
    p = _small_instances()[idx]
    H, Q = p["H"], p["Q"]
    Lam = oracle.uniformisation(p)
    assert Lam == pytest.approx(p["lam"] + p["C"] * sum(p["mu"]) + sum(p["delta"]) + 1.0, rel=1e-15)
    for s in range(oracle.num_states(p)):
        occ, q, ph = oracle.decode(p, s)
        any_feasible = False
        for a in range(H + 1):
            row = oracle.transitions(p, s, a)
            if row is None:
                continue
            any_feasible = True
            cols, probs, _ = row
            assert np.all(probs > 0.0)
            assert abs(probs.sum() - 1.0) <= 1e-15 * 4
            assert np.all(np.diff(cols) > 0)
            assert len(cols) <= 2 * H + 3
            # post-decision occupancy and queue
            o = list(occ)
            qq = q
            if a < H:
                o[a] += 1
                qq -= 1
            expect_n = 2 * sum(1 for v in o if v > 1) + sum(1 for v in o if v == 1) + (1 if qq < Q else 0) + 2
            assert len(cols) == expect_n
        assert any_feasible  # defer is always available


def test_phase_flip_law():
    """The phase bit is an autonomous two-state chain: P(CCHI->SCHI) = f/Lam and
    P(SCHI->CCHI) = (1-f)/Lam from every row, so the stationary SCHI fraction is f."""
    p = inputs.workload("tiny")
    Lam = oracle.uniformisation(p)
    for s in range(oracle.num_states(p)):
        _, _, ph = oracle.decode(p, s)
        for a in range(p["H"] + 1):
            row = oracle.transitions(p, s, a)
            if row is None:
                continue
            cols, probs, _ = row
            flip = sum(pr for c, pr in zip(cols, probs) if c % 2 != ph)
            want = (p["f"] if ph == 0 else 1.0 - p["f"]) / Lam
            assert flip == pytest.approx(want, rel=1e-14)
    a01 = p["f"] / Lam
    a10 = (1 - p["f"]) / Lam
    assert a01 / (a01 + a10) == pytest.approx(p["f"], rel=1e-14)


def test_feasibility_rule():
    p = inputs.workload("tiny")
    H, C = p["H"], p["C"]
    for s in range(oracle.num_states(p)):
        occ, q, ph = oracle.decode(p, s)
        for a in range(H):
            want = q >= 1 and occ[a] < C and (a == H - 1 or ph == 1)
            assert oracle.feasible(p, s, a) == want
        assert oracle.feasible(p, s, H)


def test_canonical_and_padded_counts():
    # The tiny workload has 1,408 feasible rows and 9,696 canonical successors; these
    # counts were obtained by an independent exhaustive count when the workload was specified.
    p = inputs.workload("tiny")
    row_ptr, col, val, R = oracle.build_csr(p)
    S, A = 640, 4
    assert len(row_ptr) == S * A + 1
    assert int(np.sum(np.isfinite(R))) == 1408
    assert row_ptr[-1] == 9696 == oracle.csr_nnz(p)
    assert oracle.csr_nnz(p, padded=True) == S * A * (2 * p["H"] + 3) == 23040
    rp2, col2, val2, R2 = oracle.build_csr(p, padded=True)
    assert np.array_equal(R, R2)
    for r in range(S * A):
        lo, hi = row_ptr[r], row_ptr[r + 1]
        lo2, hi2 = rp2[r], rp2[r + 1]
        assert hi2 - lo2 == 2 * p["H"] + 3
        n = hi - lo
        assert np.array_equal(col[lo:hi], col2[lo2:lo2 + n])
        assert np.array_equal(val[lo:hi], val2[lo2:lo2 + n])
        assert np.all(val2[lo2 + n:hi2] == 0.0)
        assert np.all(np.diff(col2[lo2:hi2]) >= 0)


def test_reward_definition_on_all_rows():
    """R(s,a) re-derived from the post-decision state by the stated formula."""
    p = inputs.make_params(2, 3, 2, 0.9, seed=11)
    H, Q = p["H"], p["Q"]
    Lam = oracle.uniformisation(p)
    for s in range(oracle.num_states(p)):
        occ, q, ph = oracle.decode(p, s)
        for a in range(H + 1):
            row = oracle.transitions(p, s, a)
            if row is None:
                continue
            o = list(occ)
            qq = q
            if a < H:
                o[a] += 1
                qq -= 1
            lost = sum(p["delta"][k] * o[k] for k in range(H)) / Lam + (p["lam"] / Lam if qq == Q else 0.0)
            want = p["w_occ"] * sum(o) + p["w_q"] * qq + p["w_loss"] * lost
            assert row[2] == pytest.approx(want, rel=1e-13, abs=1e-14)
