"""Algorithm 4's in-block iteration (VC_ITER_BLOCK) on implicit handles, against the oracle's
block iteration over the model's CSR (or_block_vi_csr_sl: consecutive blocks of `tile`
states, `passes` local Jacobi passes of the self-transition-solved backup, pinned in
test_oracle_self_loop.py), and against V*.

* One local pass is the plain self-transition sweep, bit for bit.
* k global sweeps with p local passes on blocks of B = 2(Q+1)(C+1)^h states equal the
  oracle's block iteration with tile = B and the same p within the FP32 bound below.
* Certified solves: V64 within 1e-6 relative of V*, the policy equal wherever the oracle's
  Q-gap exceeds 1e-6, with fewer global sweeps than the one-state self-transition solve.
* At full size (2.5 M states, blocks of 160 states) the certified V64 backs up within
  gamma 1e-6 at every state.
* Errors: explicit handles, bad shapes.

FP32 bound of k global sweeps of p local passes: each local pass is one self-transition
backup whose row sums take at most n + 4 roundings of terms bounded by |R|max + |V|max,
divided by 1 - gamma p_max (derivation in test_gpu_self_loop.py); the in-block corrections
add differences of the same values.  Errors of earlier passes propagate contracted, so
k p (n + 6) u (|R|max + |V|max) / (1 - gamma p_max) + 2 u |W|max bounds the distance.
"""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

from gpu_common import native_or_skip, policy_mismatches, rel_err

pytestmark = pytest.mark.gpu

U32 = 2.0**-24
MID = inputs.make_params(4, 4, 6, 0.95, seed=7)   # S = 8750; blocks of 14 (h=0), 70, 350 states
TINY = inputs.workload("tiny")                     # S = 640
_csr = {}


def _csr_of(p, key):
    if key not in _csr:
        _csr[key] = oracle.build_csr(p)
    return _csr[key]


def _seeded(S, seed, scale):
    import torch

    g = torch.Generator(device="cuda").manual_seed(seed)
    return (torch.rand(S, device="cuda", generator=g) - 0.3) * scale


def _sweeps(m, V0, k, **kw):
    V = V0.clone()
    _, _, _, st = m.value_iterate(V=V, tol=1e-30, max_sweeps=k, fp32_only=True, want_v64=False, want_pi=False,
                                  raise_on_nonconvergence=False, **kw)
    assert st["sweeps"] == k
    return V


def test_one_local_pass_is_the_self_transition_sweep_bitwise():
    native = native_or_skip()
    import torch

    for p in (TINY, MID):
        m = native.MDP.build(p, fmt="implicit")
        V0 = _seeded(m.S, 3, 60.0)
        for h in range(0, 3):
            m.set_block_iteration(h, 1)
            for k in (1, 4):
                a = _sweeps(m, V0, k, block=True)
                b = _sweeps(m, V0, k, self_loop=True)
                assert torch.equal(a, b), (h, k)
        m.close()


@pytest.mark.parametrize("h,passes", [(0, 2), (1, 3), (2, 4), (2, 2)])
@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_block_sweeps_match_the_oracle(name, h, passes):
    native = native_or_skip()
    p = TINY if name == "tiny" else MID
    rp, col, val, R = _csr_of(p, name)
    S, A = oracle.num_states(p), oracle.num_actions(p)
    m = native.MDP.build(p, fmt="implicit")
    m.set_block_iteration(h, passes)
    info = m.block_iteration_info()
    B = 2 * (p["Q"] + 1) * (p["C"] + 1) ** h
    assert info == {"inner_hosts": h, "block_states": B, "passes": passes}
    V0 = _seeded(S, 5, 40.0)
    V0h = V0.cpu().numpy().astype(np.float64)
    n = int(np.max(np.diff(rp)))
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    own = col == rows // A
    pss = np.zeros(len(rp) - 1)
    np.add.at(pss, rows[own], val[own])
    Rmax = np.abs(R[np.isfinite(R)]).max()
    for k in (1, 3):
        V = _sweeps(m, V0, k, block=True).cpu().numpy().astype(np.float64)
        Wo, _ = oracle.block_vi_csr_self_loop(S, A, rp, col, val, R, p["gamma"], B, passes, tol=1e-300,
                                              max_sweeps=k, V0=V0h, strict=False)
        vmax = max(np.abs(V0h).max(), np.abs(Wo).max())
        bound = k * passes * (n + 6) * U32 * (Rmax + vmax) / (1 - p["gamma"] * pss.max()) + 2 * U32 * vmax
        assert np.max(np.abs(V - Wo)) <= bound, (k, np.max(np.abs(V - Wo)), bound)
    m.close()


@pytest.mark.parametrize("gamma", [0.95, 0.99])
def test_block_solve_is_certified_with_fewer_sweeps(gamma):
    native = native_or_skip()
    p = inputs.make_params(4, 4, 6, gamma, seed=7)
    Vs, pis, gaps, _ = oracle.solve(p, tol=1e-12)
    m = native.MDP.build(p, fmt="implicit")
    _, _, _, st_sl = m.value_iterate(tol=1e-6, self_loop=True)
    for h, passes in ((1, 4), (2, 4), (2, 8)):
        m.set_block_iteration(h, passes)
        _, V64, pi, st = m.value_iterate(tol=1e-6, block=True)
        assert st["certified"] == 1 and st["residual64"] < 1e-6
        assert rel_err(V64.cpu().numpy(), Vs) <= 1e-6
        assert policy_mismatches(pi.cpu().numpy(), pis, gaps)[0] == 0
        assert st["sweeps"] < st_sl["sweeps"], (h, passes, st["sweeps"], st_sl["sweeps"])
    m.close()


def test_block_solve_at_full_size_every_state():
    native = native_or_skip()
    p = inputs.workload("large")
    m = native.MDP.build(p, fmt="implicit")
    info = m.block_iteration_info()
    assert info["block_states"] == 160 and info["inner_hosts"] == 1
    _, _, _, st_sl = m.value_iterate(tol=1e-6, self_loop=True, want_v64=False, want_pi=False)
    _, V64, pi, st = m.value_iterate(tol=1e-6, block=True)
    assert st["certified"] == 1 and st["residual64"] < 1e-6
    assert st["sweeps"] < st_sl["sweeps"]
    V64 = V64.cpu().numpy()
    Tv, pio, gapo = oracle.backup_all(p, V64)
    assert float(np.max(np.abs(Tv - V64))) <= p["gamma"] * 1e-6 + 1e-9
    sel = gapo > 1e-6
    assert int(np.sum(pi.cpu().numpy()[sel] != pio[sel])) == 0
    m.close()


def test_block_iteration_errors():
    native = native_or_skip()
    p = MID
    m = native.MDP.build(p, fmt="csr_f32")
    with pytest.raises(native.VcError) as e:
        m.value_iterate(tol=1e-6, block=True)
    assert e.value.code == native.VC_ERR_ARG
    with pytest.raises(native.VcError):
        m.set_block_iteration(1, 4)
    m.close()
    m = native.MDP.build(p, fmt="implicit")
    for h, passes in ((1, 0), (1, 65), (3, 2), (5, 2), (-2, 2)):
        with pytest.raises(native.VcError) as e:
            m.set_block_iteration(h, passes)
        assert e.value.code == native.VC_ERR_ARG, (h, passes)
    # a rejected shape leaves the previous one in place
    assert m.block_iteration_info()["block_states"] == 350
    m.close()


def _batch_block_states(p, threads):
    B = 2 * (p["Q"] + 1)
    h = 0
    while h < p["H"] and B * (p["C"] + 1) <= threads:
        B *= p["C"] + 1
        h += 1
    return B


@pytest.mark.parametrize("threads,passes", [(256, 3), (512, 4)])
def test_batched_block_iteration_against_the_oracle(threads, passes):
    """The batch's in-block loop (its own captured graph, blocks per instance): one local
    pass equals the batch's self-transition loop bitwise; k global sweeps of every instance
    equal the oracle's block iteration on that instance's blocks within the bound; the
    certified solve matches every optimum with fewer total sweeps than the one-state
    self-transition loop."""
    native = native_or_skip()
    import torch

    ps = [p for p in inputs.batch_params(512, seed=2) if inputs.num_states(p["H"], p["C"], p["Q"]) <= 4000][:14]
    assert {p["gamma"] for p in ps} == {0.9, 0.95, 0.99}
    b = native.Batch(ps)
    b.set_small_instances(0)  # these instances would otherwise be swept whole in one CTA each
    off = b.offsets
    V0 = _seeded(int(off[-1]), 6, 30.0)
    # one local pass: the self-transition loop, bit for bit
    b.set_block_iteration(threads, 1)
    Va, Vb = V0.clone(), V0.clone()
    b.value_iterate(V=Va, tol=1e-30, max_sweeps=3, fp32_only=True, raise_on_nonconvergence=False, block=True)
    b.value_iterate(V=Vb, tol=1e-30, max_sweeps=3, fp32_only=True, raise_on_nonconvergence=False, self_loop=True)
    assert torch.equal(Va, Vb)
    b.set_block_iteration(threads, passes)
    V0h = V0.cpu().numpy().astype(np.float64)
    for k in (1, 3):
        V = V0.clone()
        _, _, _, stats, _ = b.value_iterate(V=V, tol=1e-30, max_sweeps=k, fp32_only=True,
                                            raise_on_nonconvergence=False, block=True)
        assert all(s["sweeps"] == k for s in stats)
        V = V.cpu().numpy().astype(np.float64)
        for i, p in enumerate(ps):
            sl = slice(off[i], off[i + 1])
            rp, col, val, R = _csr_of(p, ("batch", i))
            S, A = oracle.num_states(p), oracle.num_actions(p)
            B = _batch_block_states(p, threads)
            Wo, _ = oracle.block_vi_csr_self_loop(S, A, rp, col, val, R, p["gamma"], B, passes, tol=1e-300,
                                                  max_sweeps=k, V0=V0h[sl], strict=False)
            rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
            own = col == rows // A
            pss = np.zeros(len(rp) - 1)
            np.add.at(pss, rows[own], val[own])
            n = int(np.max(np.diff(rp)))
            vmax = max(np.abs(V0h[sl]).max(), np.abs(Wo).max())
            Rmax = np.abs(R[np.isfinite(R)]).max()
            bound = k * passes * (n + 6) * U32 * (Rmax + vmax) / (1 - p["gamma"] * pss.max()) + 2 * U32 * vmax
            assert np.max(np.abs(V[sl] - Wo)) <= bound, (i, k, np.max(np.abs(V[sl] - Wo)), bound)
    _, _, _, st_sl, rc = b.value_iterate(tol=1e-6, accurate=True, self_loop=True)
    _, V64, pi, stats, rc = b.value_iterate(tol=1e-6, accurate=True, block=True)
    assert rc == native.VC_OK and all(s["certified"] == 1 for s in stats)
    V64, pi = V64.cpu().numpy(), pi.cpu().numpy()
    for i, p in enumerate(ps):
        sl = slice(off[i], off[i + 1])
        Vs, pis, gaps, _ = oracle.solve(p, tol=1e-12)
        assert np.max(np.abs(V64[sl] - Vs)) <= 5e-7 + 1e-9
        assert policy_mismatches(pi[sl], pis, gaps)[0] == 0
    assert sum(s["sweeps"] for s in stats) < sum(s["sweeps"] for s in st_sl)
    for threads, passes in ((16, 4), (1024, 4), (512, 0)):
        with pytest.raises(native.VcError) as e:
            b.set_block_iteration(threads, passes)
        assert e.value.code == native.VC_ERR_ARG
    # a rejected shape keeps the previous one: the batch still solves
    _, V64b, _, stats, rc = b.value_iterate(tol=1e-6, accurate=True, block=True)
    assert rc == native.VC_OK and all(s["certified"] == 1 for s in stats)
    b.close()


def test_batched_block_iteration_full_workload_certified():
    native = native_or_skip()
    ps = inputs.batch_params(512, seed=2)
    b = native.Batch(ps)
    _, _, _, st_sl, rc = b.value_iterate(tol=1e-6, self_loop=True)
    _, V64, pi, stats, rc = b.value_iterate(tol=1e-6, block=True)
    assert rc == native.VC_OK and all(s["certified"] == 1 for s in stats)
    assert sum(s["sweeps"] for s in stats) < sum(s["sweeps"] for s in st_sl)
    # sampled instances against the oracle's backup of every state
    off = b.offsets
    V64 = V64.cpu().numpy()
    pi = pi.cpu().numpy()
    for i in (0, 17, 101, 311, 511):
        p = ps[i]
        sl = slice(off[i], off[i + 1])
        Tv, pio, gapo = oracle.backup_all(p, V64[sl])
        assert float(np.max(np.abs(Tv - V64[sl]))) <= p["gamma"] * 1e-6 + 1e-9
        sel = gapo > 1e-6
        assert int(np.sum(pi[sl][sel] != pio[sel])) == 0
    b.close()
