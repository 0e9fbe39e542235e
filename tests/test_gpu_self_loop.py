"""FP32 sweeps with each action's self-transition solved (VC_ITER_SELF_LOOP), against the
oracle's transcription of the same iteration (pinned in test_oracle_self_loop.py) and
against V*.

* One sweep from a seeded V on every storage form equals the oracle's sweep of the same V
  within the FP32 bound below, and the explicit kernels (pipelined CSR, direct CSR, sliced
  ring, sliced direct) agree bitwise with each other, FP32 and BF16 storage, canonical and
  padded rows.
* A full solve with the flag is certified, V64 within 1e-6 relative of the oracle's V*, the
  policy equal wherever the oracle's Q-gap exceeds 1e-6, and it takes fewer FP32 sweeps
  than Eq. 18's backup on the same handle.
* A user CSR whose rows contain self-transitions: the iterate after k sweeps equals the
  oracle's CSR form of the iteration within the bound, and the solve is certified.
* The batch's self-transition loop graph against every instance's oracle sweep and optimum.
* Edge cases: a one-state MDP reaches max_a R_a / (1 - gamma) in one FP32 sweep exactly;
  rows without self-transitions give Eq. 18's sweep bit for bit.

FP32 bound of one sweep (derived from the arithmetic): the numerator R + gamma off takes at
most n + 2 roundings (n stored entries, FP32 probabilities within one rounding of the FP64
ones) of terms bounded by |R|max + |V|max; the denominator 1 - gamma p_ss >= 1 - gamma
p_max takes two; the quotient one.  So |W32 - W64| <= (n + 4) u (|R|max + |V|max) /
(1 - gamma p_max) + 2 u |W|max with u = 2^-24.
"""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

from gpu_common import native_or_skip, policy_mismatches, rel_err

pytestmark = pytest.mark.gpu

MID = inputs.make_params(4, 4, 6, 0.95, seed=7)      # S = 8750, ragged tail and slices
TINY = inputs.workload("tiny")                         # S = 640
U32 = 2.0**-24
EXPLICIT = [dict(), dict(direct=True), dict(sliced=True), dict(sliced=True, direct=True)]
_solved = {}


def _sl_sweep(m, V0):
    V = V0.clone()
    _, _, _, st = m.value_iterate(V=V, tol=1e-30, max_sweeps=1, fp32_only=True, want_v64=False, want_pi=False,
                                  raise_on_nonconvergence=False, self_loop=True)
    assert st["sweeps"] == 1
    return V


def _bound(rp, col, val, R, A, V0, W, gamma):
    S = len(rp) // A
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    own = col == rows // A
    pss = np.zeros(len(rp) - 1)
    np.add.at(pss, rows[own], val[own])
    n = int(np.max(np.diff(rp)))
    Rf = np.abs(R[np.isfinite(R)]).max()
    vmax = max(np.abs(V0).max(), np.abs(W).max())
    return (n + 4) * U32 * (Rf + vmax) / (1 - gamma * pss.max()) + 2 * U32 * np.abs(W).max()


def _seeded_V(S, seed, scale=100.0):
    import torch

    g = torch.Generator(device="cuda").manual_seed(seed)
    return torch.rand(S, device="cuda", generator=g) * scale - scale / 3


@pytest.mark.parametrize("fmt,kw", [("implicit", {})] + [("csr_f32", k) for k in EXPLICIT]
                         + [("csr_f32", dict(padded=True, sliced=True))])
@pytest.mark.parametrize("which", ["tiny", "mid"])
def test_one_sweep_matches_the_oracle(which, fmt, kw):
    native = native_or_skip()
    p = TINY if which == "tiny" else MID
    m = native.MDP.build(p, fmt=fmt, **kw)
    S = m.info()["S"]
    V0 = _seeded_V(S, 3)
    W = _sl_sweep(m, V0).cpu().numpy().astype(np.float64)
    V0h = V0.cpu().numpy().astype(np.float64)
    Wo, _, _ = oracle.value_iteration_self_loop(p, tol=1e-300, max_sweeps=1, V0=V0h, strict=False)
    rp, col, val, R = oracle.build_csr(p)
    assert np.max(np.abs(W - Wo)) <= _bound(rp, col, val, R, oracle.num_actions(p), V0h, Wo, p["gamma"])
    m.close()


@pytest.mark.parametrize("fmt,padded", [("csr_f32", False), ("csr_f32", True), ("csr_bf16", False),
                                        ("csr_bf16", True)])
@pytest.mark.parametrize("which", ["tiny", "mid"])
def test_explicit_kernels_agree_bitwise(which, fmt, padded):
    native = native_or_skip()
    import torch

    p = TINY if which == "tiny" else MID
    ms = [native.MDP.build(p, fmt=fmt, padded=padded, **k) for k in EXPLICIT]
    S = ms[0].info()["S"]
    for seed, scale in ((1, 100.0), (2, 1e-3)):
        V0 = _seeded_V(S, seed, scale)
        out = [_sl_sweep(m, V0) for m in ms]
        for o in out[1:]:
            assert torch.equal(out[0], o)
    for m in ms:
        m.close()


@pytest.mark.parametrize("fmt,kw", [("implicit", {}), ("csr_f32", {}), ("csr_f32", dict(sliced=True)),
                                    ("csr_f32", dict(padded=True, sliced=True)),
                                    ("csr_bf16", dict(padded=True, sliced=True))])
@pytest.mark.parametrize("gamma", [0.95, 0.99])
def test_solve_is_certified_with_fewer_sweeps(fmt, kw, gamma):
    native = native_or_skip()
    p = inputs.make_params(4, 4, 6, gamma, seed=7)
    if gamma not in _solved:
        _solved[gamma] = oracle.solve(p, tol=1e-12)
    Vs, pis, gaps, _ = _solved[gamma]
    m = native.MDP.build(p, fmt=fmt, **kw)
    _, V64, pi, st = m.value_iterate(tol=1e-6, self_loop=True)
    assert st["certified"] == 1 and st["residual64"] < 1e-6
    assert rel_err(V64.cpu().numpy(), Vs) <= 1e-6
    assert policy_mismatches(pi.cpu().numpy(), pis, gaps)[0] == 0
    _, _, _, st_plain = m.value_iterate(tol=1e-6)
    assert st["sweeps"] < st_plain["sweeps"]
    m.close()


@pytest.mark.parametrize("S,A,succ,seed", [(40, 3, 20, 1), (2000, 6, 9, 2)])
def test_user_csr_with_self_transitions(S, A, succ, seed):
    native = native_or_skip()
    import torch

    mdp = inputs.random_csr_mdp(S, A, max_succ=succ, seed=seed, gamma=0.97)
    rp, col, R = mdp["row_ptr"], mdp["col"], mdp["R"]
    val32 = mdp["val"].astype(np.float32)
    rows = np.repeat(np.arange(S * A), np.diff(rp))
    assert np.any(col == rows // A)  # the instance has self-transitions
    dev = "cuda"
    ms = [native.MDP.from_csr(S, A, torch.tensor(rp, device=dev), torch.tensor(col, device=dev),
                              torch.tensor(val32, device=dev), torch.tensor(R.astype(np.float32), device=dev),
                              0.97)]
    v64, R64 = val32.astype(np.float64), R.astype(np.float32).astype(np.float64)
    V0 = _seeded_V(S, 4, 10.0)
    V0h = V0.cpu().numpy().astype(np.float64)
    for k in (1, 3):
        V = V0.clone()
        ms[0].value_iterate(V=V, tol=1e-30, max_sweeps=k, fp32_only=True, want_v64=False, want_pi=False,
                            raise_on_nonconvergence=False, self_loop=True)
        Wo, _ = oracle.vi_csr_self_loop(S, A, rp, col, v64, R64, 0.97, tol=1e-300, max_sweeps=k, V0=V0h,
                                        strict=False)
        assert np.max(np.abs(V.cpu().numpy() - Wo)) <= k * _bound(rp, col, v64, R64, A, V0h, Wo, 0.97)
    Vs, _ = oracle.vi_csr(S, A, rp, col, v64, R64, 0.97, tol=1e-12)
    _, V64, _, st = ms[0].value_iterate(tol=1e-6, self_loop=True)
    assert st["certified"] == 1
    assert rel_err(V64.cpu().numpy(), Vs) <= 1e-6
    ms[0].close()


def test_batched_self_loop_against_the_oracle():
    """The batch's FP32 loop with the self-transition solved (its own captured graph): one
    sweep of every instance equals the oracle's sweep within the bound, and the certified
    solve matches each instance's optimum with fewer sweeps than Eq. 18's loop."""
    native = native_or_skip()
    ps = [p for p in inputs.batch_params(512, seed=2) if inputs.num_states(p["H"], p["C"], p["Q"]) <= 4000][:18]
    assert {p["gamma"] for p in ps} == {0.9, 0.95, 0.99}
    b = native.Batch(ps)
    off = b.offsets
    V0 = _seeded_V(int(off[-1]), 6)
    V = V0.clone()
    b.value_iterate(V=V, tol=1e-30, max_sweeps=1, fp32_only=True, raise_on_nonconvergence=False, self_loop=True)
    V, V0h = V.cpu().numpy().astype(np.float64), V0.cpu().numpy().astype(np.float64)
    for i, p in enumerate(ps):
        sl = slice(off[i], off[i + 1])
        Wo, _, _ = oracle.value_iteration_self_loop(p, tol=1e-300, max_sweeps=1, V0=V0h[sl], strict=False)
        rp, col, val, R = oracle.build_csr(p)
        assert np.max(np.abs(V[sl] - Wo)) <= _bound(rp, col, val, R, oracle.num_actions(p), V0h[sl], Wo,
                                                    p["gamma"])
    res = {}
    for flag in (False, True):
        _, V64, pi, stats, rc = b.value_iterate(tol=1e-6, accurate=True, self_loop=flag)
        assert rc == native.VC_OK and all(s["certified"] == 1 for s in stats)
        res[flag] = (V64.cpu().numpy(), pi.cpu().numpy(), stats)
    for i, p in enumerate(ps):
        sl = slice(off[i], off[i + 1])
        Vs, pis, gaps, _ = oracle.solve(p, tol=1e-12)
        V64, pi, stats = res[True]
        assert np.max(np.abs(V64[sl] - Vs)) <= 5e-7 + 1e-9
        assert policy_mismatches(pi[sl], pis, gaps)[0] == 0
        if p["gamma"] == 0.99:
            assert stats[i]["sweeps"] < res[False][2][i]["sweeps"]
    b.close()


def test_edge_cases_one_state_and_no_self_transitions():
    """A one-state MDP (every row a self-transition) reaches max_a R_a / (1 - gamma) in one
    sweep; rows without self-transitions give Eq. 18's sweep bit for bit."""
    native = native_or_skip()
    import torch

    dev = "cuda"
    g = 0.95
    Rr = np.array([0.3, 1.7, -2.0], np.float32)
    m = native.MDP.from_csr(1, 3, torch.tensor([0, 1, 2, 3], dtype=torch.int64, device=dev),
                            torch.zeros(3, dtype=torch.int32, device=dev), torch.ones(3, device=dev),
                            torch.tensor(Rr, device=dev), g)
    W = _sl_sweep(m, torch.zeros(1, device=dev)).cpu().numpy()
    assert W[0] == np.float32(np.float32(1.7) / (np.float32(1.0) - np.float32(g)))
    m.close()
    # no self-transitions: a ring of states, each row moving to the next states only
    S, A = 300, 3
    rng = np.random.default_rng(9)
    rp, col, val, R = [0], [], [], []
    for s in range(S):
        for a in range(A):
            c = sorted({(s + 1 + int(k)) % S for k in rng.integers(0, 5, size=3)})
            w = rng.random(len(c)) + 0.1
            col += c
            val += (w / w.sum()).tolist()
            rp.append(len(col))
            R.append(rng.uniform(-1, 1))
    args = (torch.tensor(rp, dtype=torch.int64, device=dev), torch.tensor(col, dtype=torch.int32, device=dev),
            torch.tensor(val, dtype=torch.float32, device=dev), torch.tensor(R, dtype=torch.float32, device=dev))
    m = native.MDP.from_csr(S, A, *args, 0.9)
    V0 = _seeded_V(S, 8, 5.0)
    Vo = torch.empty_like(V0)
    m.bellman32(V0, Vo)
    torch.cuda.synchronize()
    assert torch.equal(_sl_sweep(m, V0), Vo)
    m.close()
