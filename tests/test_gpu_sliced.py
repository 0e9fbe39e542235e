"""The sliced (SELL-C-sigma) copy of the stored matrix and its FP32 sweep.

* one sweep on the sliced copy equals the CSR sweep bitwise (values, policy, Q-gap) for
  the generated model in every stored form and for arbitrary CSR matrices (ragged rows,
  infeasible actions, A from 1 to 31, S from 1 to several windows of 4096 with a ragged
  last slice);
* the copy's size (entries incl. padding) equals a host-side recomputation of the layout
  from the oracle's CSR (sort key, slice widths) exactly;
* a full solve on the sliced copy is certified and matches the oracle within 1e-6;
* every candidate schedule (selected with vc_sweep_schedule) gives the same sweep bit for
  bit, in Eq. 18's backup and the self-transition solve;
* the autotuner's sliced candidates keep the results; invalid requests are errors.
"""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

from gpu_common import native_or_skip, policy_mismatches, rel_err

pytestmark = pytest.mark.gpu

MID = inputs.make_params(4, 4, 6, 0.95, seed=7)      # S = 8750: three windows, ragged slice
TINY = inputs.workload("tiny")                         # S = 640: one partial window
CSR_FORMS = [("csr_f32", False), ("csr_f32", True), ("csr_bf16", False), ("csr_bf16", True)]


def _sweep(m, V):
    import torch

    Vo = torch.empty_like(V)
    pi = torch.empty(V.numel(), dtype=torch.int32, device=V.device)
    gap = torch.empty_like(V)
    m.bellman32(V, Vo, pi, gap)
    torch.cuda.synchronize()
    return Vo, pi, gap


def _host_slice_rows(row_ptr, R, S, A, val=None, C=32, sigma=4096):
    """Rows (of 32 entries) of every slice of the sliced layout, recomputed on the host from
    the layout's definition: rows keep their non-zero entries; states sorted in windows by
    (feasible mask, -total length, index); per slice and action the longest feasible row."""
    row_ptr = np.asarray(row_ptr)
    if val is None:
        L = np.diff(row_ptr).reshape(S, A)
    else:
        nz = np.concatenate([[0], np.cumsum(np.asarray(val) != 0)])
        L = (nz[row_ptr[1:]] - nz[row_ptr[:-1]]).reshape(S, A)
    feas = np.asarray(R).reshape(S, A) != -np.inf
    L = np.where(feas, L, 0)
    mask = (feas[:, : min(A, 30)] * (1 << np.arange(min(A, 30)))).sum(axis=1)
    if A > 30:
        mask = mask | (feas[:, 30:].any(axis=1) << 30)
    tot = np.minimum(L.sum(axis=1), 0xFFFFF)
    order = []
    for w0 in range(0, S, sigma):
        idx = np.arange(w0, min(S, w0 + sigma))
        order.append(idx[np.lexsort((idx, -tot[idx], mask[idx]))])
    order = np.concatenate(order)
    Lo = L[order]
    pad = (-S) % C
    Lo = np.vstack([Lo, np.zeros((pad, A), dtype=Lo.dtype)])
    return Lo.reshape(-1, C, A).max(axis=1).sum(axis=1)


def _host_sliced_entries(row_ptr, R, S, A, val=None):
    return int(_host_slice_rows(row_ptr, R, S, A, val).sum()) * 32


def _host_sweep_bytes(row_ptr, R, S, A, vbytes, val=None):
    """Slab bytes (one record per slice: header, state map, R [and scale], col, val rows,
    each region rounded to 128 bytes) + record offsets + V in and out."""
    rows = _host_slice_rows(row_ptr, R, S, A, val)
    r128 = lambda x: (x + 127) // 128 * 128
    rec = 256 + 128 * A * (2 if vbytes == 2 else 1) + 128 * rows + r128(32 * vbytes * rows)
    G = len(rows)
    return int(rec.sum()) + 8 * (G + 1) + 8 * S


@pytest.mark.parametrize("fmt,padded", CSR_FORMS)
@pytest.mark.parametrize("which", ["tiny", "mid"])
def test_sliced_sweep_equals_csr_sweep(which, fmt, padded):
    native = native_or_skip()
    import torch

    p = TINY if which == "tiny" else MID
    mc = native.MDP.build(p, fmt=fmt, padded=padded, direct=True)
    ms = native.MDP.build(p, fmt=fmt, padded=padded, sliced=True)
    md = native.MDP.build(p, fmt=fmt, padded=padded, sliced=True, direct=True)
    info = ms.info()
    assert info["csr_sliced"] == 1 and info["nnz_sliced"] > 0
    assert info["csr_pipelined"] == 1 and md.info()["csr_pipelined"] == 0
    S, A = info["S"], info["A"]
    rp, col, val, R = oracle.build_csr(p, padded=padded)[:4]
    assert info["nnz_sliced"] == _host_sliced_entries(rp, R, S, A, val)
    vbytes = 2 if fmt == "csr_bf16" else 4
    assert info["sweep_bytes"] == _host_sweep_bytes(rp, R, S, A, vbytes, val)
    if padded:
        # the padded matrix's filler zeros are not stored: its sliced copy is the canonical one's
        rc, _, vc, Rc = oracle.build_csr(p, padded=False)[:4]
        assert info["nnz_sliced"] == _host_sliced_entries(rc, Rc, S, A, vc)
    g = torch.Generator(device="cuda").manual_seed(5)
    for scale in (100.0, 1e-3):
        V = torch.rand(S, device="cuda", generator=g) * scale - scale / 3
        a, b, c = _sweep(mc, V), _sweep(ms, V), _sweep(md, V)
        for x, y, z in zip(a, b, c):
            assert torch.equal(x, y) and torch.equal(x, z)
    mc.close()
    ms.close()
    md.close()


@pytest.mark.parametrize("S,A,seed", [(1, 1, 0), (7, 3, 1), (300, 5, 2), (5000, 9, 3), (9000, 31, 4),
                                      (33, 2, 5)])
def test_sliced_arbitrary_csr(S, A, seed):
    native = native_or_skip()
    import torch

    mdp = inputs.random_csr_mdp(S, A, max_succ=min(S, 12), seed=seed, gamma=0.9)
    val32 = mdp["val"].astype(np.float32)
    R32 = mdp["R"].astype(np.float32)
    dev = "cuda"
    args = (S, A, torch.tensor(mdp["row_ptr"], device=dev), torch.tensor(mdp["col"], device=dev),
            torch.tensor(val32, device=dev), torch.tensor(R32, device=dev), 0.9)
    mc = native.MDP.from_csr(*args)
    ms = native.MDP.from_csr(*args).slice()
    assert ms.info()["nnz_sliced"] == _host_sliced_entries(mdp["row_ptr"], R32, S, A)
    g = torch.Generator(device="cuda").manual_seed(seed)
    V = torch.rand(S, device=dev, generator=g) * 10
    ref = _sweep(mc, V)
    for x, y in zip(ref, _sweep(ms, V)):
        assert torch.equal(x, y)
    # every schedule the autotuner may pick (pipelined / direct, CSR / sliced), each one
    for k in range(ms.schedules()):
        ms.use_schedule(k)
        for x, y in zip(ref, _sweep(ms, V)):
            assert torch.equal(x, y), k
    ms.autotune(reps=2)
    for x, y in zip(ref, _sweep(ms, V)):
        assert torch.equal(x, y)
    # full certified solve on the sliced copy against the oracle on the same FP32 matrix
    Vo, _ = oracle.vi_csr(S, A, mdp["row_ptr"], mdp["col"], val32.astype(np.float64), R32.astype(np.float64), 0.9,
                          tol=1e-12)
    pio, gapo = oracle.policy_csr(S, A, mdp["row_ptr"], mdp["col"], val32.astype(np.float64),
                                  R32.astype(np.float64), 0.9, Vo)
    _, V64, pi, st = ms.value_iterate(tol=1e-8)
    assert st["certified"] == 1
    assert np.max(np.abs(V64.cpu().numpy() - Vo)) <= 1e-6 * max(1.0, np.max(np.abs(Vo)))
    assert policy_mismatches(pi.cpu().numpy(), pio, gapo)[0] == 0
    mc.close()
    ms.close()


@pytest.mark.parametrize("fmt,padded", [("csr_f32", False), ("csr_bf16", True)])
def test_sliced_solve_matches_oracle(fmt, padded):
    native = native_or_skip()
    p = MID
    m = native.MDP.build(p, fmt=fmt, padded=padded, sliced=True)
    _, V64, pi, st = m.value_iterate(tol=1e-6)
    assert st["certified"] == 1
    Vs, pis, gaps, _ = oracle.solve(p, tol=1e-12)
    assert rel_err(V64.cpu().numpy(), Vs) <= 1e-6
    assert policy_mismatches(pi.cpu().numpy(), pis, gaps)[0] == 0
    # same iterate and sweep count as the CSR handle (bitwise-equal sweeps)
    mc = native.MDP.build(p, fmt=fmt, padded=padded)
    V1, _, _, s1 = mc.value_iterate(tol=1e-6, fp32_only=True)
    V2, _, _, s2 = m.value_iterate(tol=1e-6, fp32_only=True)
    import torch

    assert s1["sweeps"] == s2["sweeps"] and torch.equal(V1, V2)
    m.close()
    mc.close()


@pytest.mark.parametrize("fmt,padded", CSR_FORMS)
def test_every_schedule_is_bitwise_equal(fmt, padded):
    """Every candidate schedule (CSR tilings, ring sweep launch shapes and tile sizes,
    direct kernels): one sweep equal bit for bit to the
    direct CSR kernel's, and the self-transition solve's FP32 iterate and sweep count equal
    to the CSR handle's."""
    native = native_or_skip()
    import torch

    mc = native.MDP.build(MID, fmt=fmt, padded=padded, direct=True)
    ms = native.MDP.build(MID, fmt=fmt, padded=padded, sliced=True)
    g = torch.Generator(device="cuda").manual_seed(11)
    V = torch.rand(ms.S, device="cuda", generator=g) * 80 - 20
    ref = _sweep(mc, V)
    Vr, _, _, sr = mc.value_iterate(tol=1e-6, fp32_only=True, self_loop=True)
    n = ms.schedules()
    rep_kinds = set()
    for k in range(n):
        ms.use_schedule(k)
        info = ms.info()
        rep_kinds.add((info["csr_sliced"], info["csr_pipelined"]))
        for x, y in zip(ref, _sweep(ms, V)):
            assert torch.equal(x, y), k
        Vk, _, _, sk = ms.value_iterate(tol=1e-6, fp32_only=True, self_loop=True)
        assert sk["sweeps"] == sr["sweeps"] and torch.equal(Vk, Vr), k
    assert rep_kinds == {(0, 0), (0, 1), (1, 0), (1, 1)}
    # the autotuner's table lists the same candidates in the same order
    ms.autotune(reps=1)
    rows = ms.autotune_report().strip().splitlines()[1:]
    assert len(rows) == n
    with pytest.raises(native.VcError):
        ms.use_schedule(n)
    mc.close()
    ms.close()


def test_autotune_with_sliced_candidates_keeps_results():
    native = native_or_skip()
    import torch

    m = native.MDP.build(MID, fmt="csr_f32", padded=True, sliced=True)
    V = torch.rand(m.S, device="cuda") * 50
    ref = _sweep(m, V)
    us = m.autotune(reps=3)
    rep = m.autotune_report().strip().splitlines()
    assert us > 0 and sum(1 for r in rep if r.startswith("sliced-direct")) == 3
    assert sum(1 for r in rep if r.startswith("sliced-pipelined")) >= 3
    assert any(r.startswith("sliced-pipelined") for r in rep)
    for x, y in zip(ref, _sweep(m, V)):
        assert torch.equal(x, y)
    m.close()


def test_sliced_errors():
    native = native_or_skip()
    import torch

    with pytest.raises(native.VcError):
        native.MDP.build(TINY, fmt="implicit", sliced=True)
    mi = native.MDP.build(TINY, fmt="implicit")
    with pytest.raises(native.VcError):
        mi.slice()
    with pytest.raises(native.VcError):
        mi.schedules()
    mi.close()
    S, A = 40, 32
    mdp = inputs.random_csr_mdp(S, A, max_succ=8, seed=9, gamma=0.9)
    m = native.MDP.from_csr(S, A, torch.tensor(mdp["row_ptr"], device="cuda"), torch.tensor(mdp["col"], device="cuda"),
                            torch.tensor(mdp["val"].astype(np.float32), device="cuda"),
                            torch.tensor(mdp["R"].astype(np.float32), device="cuda"), 0.9)
    with pytest.raises(native.VcError, match="A <= 31"):
        m.slice()
    m.close()


def test_sliced_user_bf16_matrix_certified_on_its_own_values():
    """A user CSR in BF16 with its FP32 row scales (the oracle's renormalised BF16 form of the
    mid instance): the sliced sweep equals the CSR sweep bitwise, and a full solve with no
    model certifies against the stored values, matching the oracle run on that matrix."""
    native = native_or_skip()
    import torch

    p = MID
    rp, col, val, R = oracle.build_csr(p)
    bits, eff, scale = oracle.bf16_renormalised(rp, val, len(R))
    S, A = oracle.num_states(p), oracle.num_actions(p)
    R32 = R.astype(np.float32)
    dev = "cuda"
    vb = torch.tensor(bits.view(np.int16), device=dev).view(torch.bfloat16)
    args = (S, A, torch.tensor(rp, device=dev), torch.tensor(col, device=dev), vb, torch.tensor(R32, device=dev),
            p["gamma"])
    kw = dict(row_scale=torch.tensor(scale, device=dev))
    mc = native.MDP.from_csr(*args, **kw)
    ms = native.MDP.from_csr(*args, **kw).slice()
    assert ms.info()["nnz_sliced"] == _host_sliced_entries(rp, R32, S, A)
    V = torch.rand(S, device=dev) * 40
    for x, y in zip(_sweep(mc, V), _sweep(ms, V)):
        assert torch.equal(x, y)
    Vb, _ = oracle.vi_csr(S, A, rp, col, eff, R32.astype(np.float64), p["gamma"], tol=1e-12)
    pib, gapb = oracle.policy_csr(S, A, rp, col, eff, R32.astype(np.float64), p["gamma"], Vb)
    _, V64, pi, st = ms.value_iterate(tol=1e-6, accurate=True)
    assert st["certified"] == 1
    assert np.max(np.abs(V64.cpu().numpy() - Vb)) <= 5e-7 + 1e-9
    assert policy_mismatches(pi.cpu().numpy(), pib, gapb)[0] == 0
    mc.close()
    ms.close()
