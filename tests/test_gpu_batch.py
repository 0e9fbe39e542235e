"""Batched solves (vc_value_iterate_batch) against the oracle and the single-instance path.

* a batch of small uneven instances solved in accuracy mode: every instance's V64 within
  tol / 2 = 5e-7 of the oracle's optimum (so within 1e-6 relative), its policy equal where
  the oracle's gap exceeds 1e-6, and its FP32 iterate and sweep count bitwise equal to the
  single-instance implicit solve (same arithmetic, same per-instance termination); the
  single-instance accuracy mode meets the same bound;
* the batched workload (512 instances, 72 ... 436,982 states, gamma in {0.9, 0.95, 0.99})
  in accuracy mode: every instance certified with FP64 residual below
  1e-6 (1 - gamma) / (2 gamma); the oracle's own backup of EVERY state of V64 is within
  that residual and the policy equals its argmax wherever the gap exceeds 1e-6; the
  smallest instances are compared with full oracle solves;
* after an FP32 loop stopped early, the refinement's policy-improvement rounds certify the
  instances in different rounds, skipping the certified ones, and every instance still
  ends at the oracle's optimum;
* every schedule the autotuner may pick gives the same iterates.
"""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

from gpu_common import native_or_skip, policy_mismatches, rel_err

pytestmark = pytest.mark.gpu


def _small_instances(k=16, smax=3000):
    out = [p for p in inputs.batch_params(512, seed=2) if inputs.num_states(p["H"], p["C"], p["Q"]) <= smax]
    return out[:k]


def test_small_batch_matches_oracle_and_single_instance_solves():
    native = native_or_skip()
    ps = _small_instances()
    assert len(ps) == 16
    b = native.Batch(ps)
    V, V64, pi, stats, rc = b.value_iterate(tol=1e-6, accurate=True)
    assert rc == native.VC_OK
    V, V64, pi = V.cpu().numpy(), V64.cpu().numpy(), pi.cpu().numpy()
    off = b.offsets
    for i, p in enumerate(ps):
        sl = slice(off[i], off[i + 1])
        g = p["gamma"]
        assert stats[i]["certified"] == 1
        assert stats[i]["residual64"] < 1e-6 * (1 - g) / (2 * g)
        Vs, pis, gaps, _ = oracle.solve(p, tol=1e-12)
        assert np.max(np.abs(V64[sl] - Vs)) <= 5e-7 + 1e-9
        assert rel_err(V64[sl], Vs) <= 1e-6
        bad, _ = policy_mismatches(pi[sl], pis, gaps)
        assert bad == 0
        m = native.MDP.build(p, fmt="implicit")
        V1, _, _, st1 = m.value_iterate(tol=1e-6, fp32_only=True)
        assert st1["sweeps"] == stats[i]["sweeps"]
        assert np.array_equal(V1.cpu().numpy(), V[sl])
        _, V1_64, _, st2 = m.value_iterate(tol=1e-6, accurate=True)
        assert st2["certified"] == 1
        assert np.max(np.abs(V1_64.cpu().numpy() - Vs)) <= 5e-7 + 1e-9
        m.close()
    b.close()


def test_refinement_rounds_skip_certified_instances():
    """The FP32 loop stopped after a few sweeps leaves policies far from optimal, so the
    refinement runs several policy-improvement rounds and the instances certify in
    different rounds (stats "rounds"); later rounds skip the instances already certified.
    Every instance must still end at the oracle's optimum, each certified instance's values
    staying as its certifying round left them."""
    native = native_or_skip()
    ps = _small_instances()
    b = native.Batch(ps)
    V, V64, pi, stats, rc = b.value_iterate(tol=1e-6, max_sweeps=8, accurate=True, raise_on_nonconvergence=False)
    assert rc == native.VC_OK
    rounds = [s["rounds"] for s in stats]
    assert min(rounds) >= 1 and max(rounds) > min(rounds), rounds  # some instances were skipped
    V64, pi = V64.cpu().numpy(), pi.cpu().numpy()
    off = b.offsets
    for i, p in enumerate(ps):
        sl = slice(off[i], off[i + 1])
        g = p["gamma"]
        assert stats[i]["certified"] == 1 and stats[i]["termination"] == 2
        assert stats[i]["residual64"] < 1e-6 * (1 - g) / (2 * g)
        Vs, pis, gaps, _ = oracle.solve(p, tol=1e-12)
        assert np.max(np.abs(V64[sl] - Vs)) <= 5e-7 + 1e-9, i
        bad, _ = policy_mismatches(pi[sl], pis, gaps)
        assert bad == 0, i
    # FP32-only solves report no refinement round
    _, _, _, st32, _ = b.value_iterate(tol=1e-6, fp32_only=True)
    assert all(s["rounds"] == 0 for s in st32)
    b.close()


def test_batched_workload_all_certified_with_every_state_backed_up_by_the_oracle():
    native = native_or_skip()
    ps = inputs.batch_params(512, seed=2)
    sizes = np.array([inputs.num_states(p["H"], p["C"], p["Q"]) for p in ps])
    assert sizes.min() >= 72 and sizes.max() <= 436_982
    b = native.Batch(ps)
    assert b.total == int(sizes.sum())
    V, V64, pi, stats, rc = b.value_iterate(tol=1e-6, accurate=True)
    assert rc == native.VC_OK
    r_target = np.array([1e-6 * (1 - p["gamma"]) / (2 * p["gamma"]) for p in ps])
    assert all(s["certified"] == 1 and s["residual64"] < r for s, r in zip(stats, r_target))
    V64, pi = V64.cpu().numpy(), pi.cpu().numpy()
    off = b.offsets
    # every state of every instance (17.4 M in all): the oracle's own backup of the certified
    # V64 is within the instance's certified residual, and the policy is its argmax wherever
    # the oracle's Q-gap exceeds 1e-6
    for i, p in enumerate(ps):
        sl = slice(off[i], off[i + 1])
        Vi, pii = V64[sl], pi[sl]
        Tv, pio, gapo = oracle.backup_all(p, Vi)
        worst = float(np.max(np.abs(Tv - Vi)))
        assert worst <= r_target[i] + 1e-10, (i, worst, r_target[i])
        sel = gapo > 1e-6
        assert int(np.sum(pii[sel] != pio[sel])) == 0, i
    # the smallest instances against full oracle solves
    for i in np.argsort(sizes)[:3]:
        sl = slice(off[i], off[i + 1])
        Vs, pis, gaps, _ = oracle.solve(ps[i], tol=1e-12)
        assert rel_err(V64[sl], Vs) <= 1e-6
        assert policy_mismatches(pi[sl], pis, gaps)[0] == 0
    # the per-instance sweep counts follow the discount: gamma = 0.99 needs the most
    sw = np.array([s["sweeps"] for s in stats])
    gam = np.array([p["gamma"] for p in ps])
    assert np.median(sw[gam == 0.99]) > np.median(sw[gam == 0.95]) > np.median(sw[gam == 0.9])
    b.close()


def test_batch_autotune_keeps_results():
    native = native_or_skip()
    ps = _small_instances(k=40, smax=20000)
    b = native.Batch(ps)
    Va, _, _, sa, _ = b.value_iterate(tol=1e-6, fp32_only=True)
    ms = b.autotune(sweeps=10)
    assert ms > 0 and len(b.autotune_report().strip().splitlines()) == 1 + 6 * 3  # header + tiles x CTAs
    Vb, _, _, sb, _ = b.value_iterate(tol=1e-6, fp32_only=True)
    assert [s["sweeps"] for s in sa] == [s["sweeps"] for s in sb]
    import torch

    assert torch.equal(Va, Vb)
    b.close()
