"""Explicit MDPs with more than 32 actions per state (the warp-per-state CSR sweep, whose
row sums are warp-reduced instead of one lane per row), through vc_build_mdp_csr, against
the FP64 oracle's CSR routines on the same stored values.

* One FP32 sweep from a seeded V, Eq. 18's backup: values within the FP32 bound of one
  sweep below; argmax equal to the oracle's wherever its Q-gap exceeds twice that bound.
* One FP32 sweep with each action's self-transition solved (the rows hold
  self-transitions): values within the same bound divided by 1 - gamma p_max.
* Full solves with both backups: certified, V64 within 1e-6 relative (absolute below 1)
  of the oracle's optimum of the stored matrix, policy equal wherever the oracle's Q-gap
  exceeds 1e-6.
* FP32 probabilities, and BF16 probabilities with their FP32 row scales (the oracle's
  renormalised form); a second run is bitwise equal to the first; the sliced copy, limited
  to 31 actions, is refused.

FP32 bound of one sweep (derived from the arithmetic, any summation order): a row of n
stored entries takes at most n + 2 roundings of terms bounded by |R|max + |V|max (the
probabilities of an FP32 row lie within one rounding of the values the oracle reads, a
BF16 row adds the scale's product), so |Q32 - Q64| <= (n + 4) u (|R|max + |V|max), and
with the self-transition solved the division by 1 - gamma p_ss >= 1 - gamma p_max widens
that by its reciprocal plus two roundings of the quotient, u = 2^-24.
"""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

from gpu_common import native_or_skip, policy_mismatches

pytestmark = pytest.mark.gpu

U32 = 2.0**-24
GAMMA = 0.9
# (S, A, most successors per row, seed): A = 33 (one past a warp), 40, 64 (two warps)
CASES = [(300, 33, 12, 1), (200, 40, 40, 2), (150, 64, 20, 3)]


def _mdp(S, A, succ, seed, dtype):
    mdp = inputs.random_csr_mdp(S, A, max_succ=succ, seed=seed, gamma=GAMMA)
    rp, col, R = mdp["row_ptr"], mdp["col"], mdp["R"]
    R32 = R.astype(np.float32)
    if dtype == "f32":
        v32 = mdp["val"].astype(np.float32)
        return rp, col, R32, v32, None, v32.astype(np.float64)
    bits, eff, scale = oracle.bf16_renormalised(rp, mdp["val"], S * A)
    return rp, col, R32, bits, scale, eff


def _handle(native, S, A, rp, col, R32, v, scale):
    import torch

    dev = "cuda"
    if scale is None:
        vt = torch.tensor(v, device=dev)
        kw = {}
    else:
        vt = torch.tensor(v.view(np.int16), device=dev).view(torch.bfloat16)
        kw = dict(row_scale=torch.tensor(scale, device=dev))
    return native.MDP.from_csr(S, A, torch.tensor(rp, device=dev), torch.tensor(col, device=dev), vt,
                               torch.tensor(R32, device=dev), GAMMA, **kw)


def _pss(rp, col, val, A):
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    own = col == rows // A
    pss = np.zeros(len(rp) - 1)
    np.add.at(pss, rows[own], val[own])
    return pss


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("S,A,succ,seed", CASES)
def test_wide_rows_one_sweep_against_the_oracle(S, A, succ, seed, dtype):
    native = native_or_skip()
    import torch

    rp, col, R32, v, scale, eff = _mdp(S, A, succ, seed, dtype)
    R64 = R32.astype(np.float64)
    pss = _pss(rp, col, eff, A)
    assert np.count_nonzero(pss) > S // 4  # self-transitions present in many rows
    m = _handle(native, S, A, rp, col, R32, v, scale)
    assert m.info()["A"] == A
    g = torch.Generator(device="cuda").manual_seed(seed)
    V0 = (torch.rand(S, device="cuda", generator=g) - 0.5) * 20
    V0h = V0.cpu().numpy().astype(np.float64)
    n = int(np.max(np.diff(rp)))
    Rmax = float(np.abs(R64[np.isfinite(R64)]).max())

    # Eq. 18's backup, with the argmax and Q-gap outputs
    Vo = torch.empty_like(V0)
    pi = torch.empty(S, dtype=torch.int32, device="cuda")
    gap = torch.empty_like(V0)
    m.bellman32(V0, Vo, pi, gap)
    W, _ = oracle.vi_csr(S, A, rp, col, eff, R64, GAMMA, tol=1e-300, max_sweeps=1, V0=V0h, strict=False)
    pio, gapo = oracle.policy_csr(S, A, rp, col, eff, R64, GAMMA, V0h)
    bound = (n + 4) * U32 * (Rmax + np.abs(V0h).max())
    assert np.max(np.abs(Vo.cpu().numpy() - W)) <= bound
    bad, checked = policy_mismatches(pi.cpu().numpy(), pio, gapo, min_gap=2 * bound)
    assert bad == 0 and checked > S // 2
    g32 = gap.cpu().numpy()
    fin = np.isfinite(gapo)
    assert np.array_equal(np.isfinite(g32), fin)
    assert np.all(np.abs(g32[fin] - gapo[fin]) <= 2 * bound + U32 * np.abs(gapo[fin]))

    # the same sweep with each action's self-transition solved
    V = V0.clone()
    m.value_iterate(V=V, tol=1e-30, max_sweeps=1, fp32_only=True, want_v64=False, want_pi=False,
                    raise_on_nonconvergence=False, self_loop=True)
    Ws, _ = oracle.vi_csr_self_loop(S, A, rp, col, eff, R64, GAMMA, tol=1e-300, max_sweeps=1, V0=V0h, strict=False)
    bound_sl = bound / (1 - GAMMA * pss.max()) + 2 * U32 * np.abs(Ws).max()
    assert np.max(np.abs(V.cpu().numpy() - Ws)) <= bound_sl
    m.close()


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("S,A,succ,seed", CASES)
def test_wide_rows_solve_against_the_oracle(S, A, succ, seed, dtype):
    native = native_or_skip()
    import torch

    rp, col, R32, v, scale, eff = _mdp(S, A, succ, seed, dtype)
    R64 = R32.astype(np.float64)
    Vs, _ = oracle.vi_csr(S, A, rp, col, eff, R64, GAMMA, tol=1e-13)
    pis, gaps = oracle.policy_csr(S, A, rp, col, eff, R64, GAMMA, Vs)
    m = _handle(native, S, A, rp, col, R32, v, scale)
    scale_v = np.maximum(np.abs(Vs), 1.0)
    runs = []
    for sl in (False, True):
        V, V64, pi, st = m.value_iterate(tol=1e-6, accurate=True, self_loop=sl)
        assert st["certified"] == 1 and st["residual64"] < 1e-6
        V64h = V64.cpu().numpy()
        assert np.max(np.abs(V64h - Vs) / scale_v) <= 1e-6, sl
        assert policy_mismatches(pi.cpu().numpy(), pis, gaps)[0] == 0, sl
        runs.append((V, V64, pi, st["sweeps"]))
    # a second run of the Eq. 18 solve is bitwise the first
    V, V64, pi, st = m.value_iterate(tol=1e-6, accurate=True)
    assert torch.equal(V, runs[0][0]) and torch.equal(V64, runs[0][1]) and torch.equal(pi, runs[0][2])
    assert st["sweeps"] == runs[0][3]
    # the sliced copy holds at most 31 actions
    with pytest.raises(native.VcError) as e:
        m.slice()
    assert e.value.code == native.VC_ERR_ARG
    m.close()
