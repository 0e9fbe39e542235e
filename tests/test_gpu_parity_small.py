"""GPU parity against the FP64 oracle on instances the oracle solves in seconds.

Tolerances (stated by the workload and derived in the design notes):
  * certified FP64 values V64: |V64 - V*| <= 1e-6 |V*| elementwise;
  * policy: equal wherever the oracle's FP64 Q-gap exceeds 1e-6;
  * FP32 iterates: see fp32_bound below (contraction bound from the stopping residual,
    rounding accumulated over 1/(1-gamma) sweeps, and for stored FP32 probabilities the
    row-sum defect of at most 2^-24).
  * CSR structure (row_ptr, col) bit-exact; FP32 values within one FP32 rounding of the
    FP64 probability; BF16 bit patterns equal to nearest-even rounding of it.
"""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

from gpu_common import native_or_skip, policy_mismatches, rel_err

pytestmark = pytest.mark.gpu

FORMS = [("implicit", False), ("csr_f32", False), ("csr_f32", True), ("csr_bf16", False), ("csr_bf16", True)]

_ref_cache = {}


def reference(p, key):
    if key not in _ref_cache:
        _ref_cache[key] = oracle.solve(p, tol=1e-12)
    return _ref_cache[key]


# H=4, C=4, Q=6: S = 8750 states, 34.2 blocks of 256 -> a ragged tail; A = 5
MID = inputs.make_params(4, 4, 6, 0.95, seed=7)


@pytest.mark.parametrize("fmt,padded", FORMS)
@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_value_iteration_matches_oracle(name, fmt, padded):
    native = native_or_skip()
    p = inputs.workload("tiny") if name == "tiny" else MID
    Vs, pis, gaps, _ = reference(p, name)
    m = native.MDP.build(p, fmt=fmt, padded=padded)
    info = m.info()
    assert info["S"] == oracle.num_states(p)
    assert info["nnz_logical"] == oracle.csr_nnz(p)
    V, V64, pi, st = m.value_iterate(tol=1e-6)
    V64 = V64.cpu().numpy()
    pi = pi.cpu().numpy()
    assert st["certified"] == 1 and st["residual64"] < 1e-6
    assert rel_err(V64, Vs) <= 1e-6
    bad, n = policy_mismatches(pi, pis, gaps)
    assert bad == 0 and n > 0
    if fmt != "csr_bf16":
        V = V.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(V - Vs)) <= fp32_bound(p["gamma"], st["residual"], np.max(np.abs(Vs)),
                                                   stored=fmt != "implicit")


def fp32_bound(gamma, residual, vmax, stored):
    """Distance of the FP32 iterate from V*: gamma/(1-gamma) * (stopping residual) from the
    contraction, plus 2 ulp(|V|max) of rounding per sweep accumulated over 1/(1-gamma)
    sweeps, plus (stored FP32 probabilities) the row-sum defect <= 2^-24 times gamma |V|max
    amplified by 1/(1-gamma)."""
    ulp = np.spacing(np.float32(vmax)).astype(np.float64)
    b = gamma / (1 - gamma) * residual + 2 * ulp / (1 - gamma)
    if stored:
        b += gamma * 2.0**-24 * vmax / (1 - gamma)
    return b


@pytest.mark.parametrize("fmt,padded", FORMS[1:])
def test_csr_structure_matches_oracle(fmt, padded):
    native = native_or_skip()
    p = MID
    m = native.MDP.build(p, fmt=fmt, padded=padded)
    row_ptr, col, val, scale, R = (t.cpu().numpy() if t is not None else None for t in m.export_csr())
    o_rp, o_col, o_val, o_R = oracle.build_csr(p, padded=padded)
    assert np.array_equal(row_ptr, o_rp)
    assert np.array_equal(col, o_col)
    feas = np.isfinite(o_R)
    assert np.array_equal(np.isfinite(R), feas)
    assert np.all(np.abs(R[feas] - o_R[feas]) <= np.abs(o_R[feas]) * 2**-23 + 1e-6)
    if fmt == "csr_f32":
        # every stored value is the round-to-nearest FP32 of the oracle's FP64 probability
        assert np.array_equal(val, o_val.astype(np.float32))
    else:
        bits = val.view(np.uint16)
        o_bits, _, o_scale = oracle.bf16_renormalised(o_rp, o_val, len(o_R))
        assert np.array_equal(bits, o_bits)
        assert np.array_equal(scale[feas], o_scale[feas])


def test_bf16_fp32_iterate_matches_oracle_on_the_bf16_matrix():
    """The BF16 sweeps solve the renormalised BF16 MDP: their FP32 fixed point matches the
    oracle run on that same matrix; the certified V64 matches the exact-P oracle."""
    native = native_or_skip()
    p = MID
    rp, col, val, R = oracle.build_csr(p)
    _, eff, _ = oracle.bf16_renormalised(rp, val, len(R))
    S, A = oracle.num_states(p), oracle.num_actions(p)
    Vb, _ = oracle.vi_csr(S, A, rp, col, eff, R.astype(np.float32).astype(np.float64), p["gamma"], tol=1e-11)
    m = native.MDP.build(p, fmt="csr_bf16")
    V, V64, pi, st = m.value_iterate(tol=1e-6)
    V32 = V.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(V32 - Vb)) <= fp32_bound(p["gamma"], st["residual"], np.max(np.abs(Vb)), stored=True)
    Vs, _, _, _ = reference(p, "mid")
    assert rel_err(V64.cpu().numpy(), Vs) <= 1e-6
    # the modelling error of BF16 storage itself, stated: exact-P vs BF16-P optimum
    model_err = rel_err(Vb, Vs)
    assert model_err < 5e-2


@pytest.mark.parametrize("fmt", ["implicit", "csr_f32"])
def test_extract_policy_and_bellman64(fmt):
    native = native_or_skip()
    import torch

    p = MID
    Vs, pis, gaps, _ = reference(p, "mid")
    m = native.MDP.build(p, fmt=fmt)
    # FP32 policy from the FP32 image of V*: equal where the gap is well above FP32 noise
    pi32, gap32 = m.extract_policy(torch.tensor(Vs, dtype=torch.float32, device="cuda"))
    bad, _ = policy_mismatches(pi32.cpu().numpy(), pis, gaps, min_gap=1e-3)
    assert bad == 0
    # FP64 backup of a perturbed V against one-state oracle backups
    g = np.random.default_rng(1)
    Vp = Vs + g.normal(0, 0.5, len(Vs))
    out, pi64, gap64, res = m.bellman64(torch.tensor(Vp, dtype=torch.float64, device="cuda"))
    out = out.cpu().numpy()
    pi64 = pi64.cpu().numpy()
    worst = 0.0
    for s in g.choice(len(Vs), 400, replace=False):
        b, a, gp = oracle.backup(p, Vp, int(s))
        assert abs(out[s] - b) <= 1e-12 * abs(b) + 1e-12
        if gp > 1e-9:
            assert pi64[s] == a
        worst = max(worst, abs(b - Vp[s]))
    assert res >= worst - 1e-12


@pytest.mark.parametrize("fmt", ["implicit", "csr_bf16"])
def test_policy_evaluation_matches_dense_solve(fmt):
    native = native_or_skip()
    import torch

    p = inputs.workload("tiny")
    pi = oracle.greedy_policy(p)
    Vd = oracle.policy_eval_dense(p, pi)
    m = native.MDP.build(p, fmt=fmt)
    V, n = m.evaluate_policy(torch.tensor(pi, device="cuda"), tol=1e-12)
    assert rel_err(V.cpu().numpy(), Vd) <= 1e-9
    assert n > 10


def test_greedy_never_beats_the_gpu_optimum():
    native = native_or_skip()
    import torch

    p = inputs.workload("tiny")
    m = native.MDP.build(p, fmt="implicit")
    _, V64, _, st = m.value_iterate(tol=1e-6)
    Vg, _ = m.evaluate_policy(torch.tensor(oracle.greedy_policy(p), device="cuda"), tol=1e-12)
    # V64 is within gamma/(1-gamma) * 1e-6 of V*
    assert np.all(Vg.cpu().numpy() <= V64.cpu().numpy() + 19 * 1e-6 + 1e-9)


def test_deterministic_and_resumable():
    """Two runs are bitwise equal; stopping after k sweeps and warm-starting from the
    iterate reproduces the uninterrupted run bitwise (Jacobi order is fixed)."""
    native = native_or_skip()
    import torch

    p = MID
    m = native.MDP.build(p, fmt="csr_f32")
    Va, _, _, sa = m.value_iterate(tol=1e-6, fp32_only=True)
    Vb, _, _, sb = m.value_iterate(tol=1e-6, fp32_only=True)
    assert torch.equal(Va, Vb) and sa["sweeps"] == sb["sweeps"]
    k = 37
    Vk, _, _, sk = m.value_iterate(tol=1e-6, max_sweeps=k, fp32_only=True, raise_on_nonconvergence=False)
    assert sk["sweeps"] == k and sk["status"] == native.VC_ERR_NOT_CONVERGED
    V0 = torch.zeros_like(Va)
    out = torch.empty_like(Va)
    cur = V0
    for _ in range(k):
        m.bellman32(cur, out)
        cur, out = out, cur
    assert torch.equal(cur, Vk)


def test_one_state_closed_form_and_errors():
    native = native_or_skip()
    import torch

    dev = "cuda"
    # one state, three self-looping actions: V = max R / (1 - gamma)
    rp = torch.tensor([0, 1, 2, 3], dtype=torch.int64, device=dev)
    col = torch.zeros(3, dtype=torch.int32, device=dev)
    val = torch.ones(3, dtype=torch.float32, device=dev)
    R = torch.tensor([0.5, 2.0, -1.0], dtype=torch.float32, device=dev)
    m = native.MDP.from_csr(1, 3, rp, col, val, R, 0.9)
    V, V64, pi, st = m.value_iterate(tol=1e-9)
    assert abs(V64.item() - 20.0) < 1e-8 and pi.item() == 1
    # a row that does not sum to one
    with pytest.raises(native.VcError) as e:
        native.MDP.from_csr(1, 3, rp, col, val * 0.5, R, 0.9)
    assert e.value.code == native.VC_ERR_NOT_STOCHASTIC
    # a state without any feasible action
    Rinf = torch.full((3,), float("-inf"), dtype=torch.float32, device=dev)
    with pytest.raises(native.VcError) as e:
        native.MDP.from_csr(1, 3, rp, col, val, Rinf, 0.9)
    assert e.value.code == native.VC_ERR_NO_FEASIBLE_ACTION
    # column out of range
    with pytest.raises(native.VcError) as e:
        native.MDP.from_csr(1, 3, rp, col + 1, val, R, 0.9)
    assert e.value.code == native.VC_ERR_ARG
    # bad model parameters
    bad = dict(inputs.workload("tiny"))
    bad["gamma"] = 1.0
    with pytest.raises(native.VcError) as e:
        native.MDP.build(bad)
    assert e.value.code == native.VC_ERR_ARG
    bad = dict(inputs.workload("tiny"))
    bad["H"] = 0
    with pytest.raises(native.VcError):
        native.MDP.build(bad)
    # infeasible policy for evaluation
    m2 = native.MDP.build(inputs.workload("tiny"))
    pi_bad = torch.zeros(640, dtype=torch.int32, device=dev)  # action 0 needs SCHI and a task
    with pytest.raises(native.VcError) as e:
        m2.evaluate_policy(pi_bad)
    assert e.value.code == native.VC_ERR_ARG
    # max_sweeps exhausted
    _, _, _, st = m2.value_iterate(tol=1e-6, max_sweeps=3, fp32_only=True, raise_on_nonconvergence=False)
    assert st["status"] == native.VC_ERR_NOT_CONVERGED and st["sweeps"] == 3


@pytest.mark.parametrize("seed", range(4))
def test_random_explicit_mdp(seed):
    """Arbitrary CSR (ragged rows, infeasible actions, A not a power of two)."""
    native = native_or_skip()
    import torch

    S = [1, 7, 300, 1000][seed]
    A = [1, 3, 5, 9][seed]
    mdp = inputs.random_csr_mdp(S, A, max_succ=min(S, 12), seed=seed, gamma=0.9)
    val32 = mdp["val"].astype(np.float32)
    R32 = mdp["R"].astype(np.float32)
    Vo, _ = oracle.vi_csr(S, A, mdp["row_ptr"], mdp["col"], val32.astype(np.float64), R32.astype(np.float64), 0.9,
                          tol=1e-12)
    pio, gapo = oracle.policy_csr(S, A, mdp["row_ptr"], mdp["col"], val32.astype(np.float64),
                                  R32.astype(np.float64), 0.9, Vo)
    dev = "cuda"
    m = native.MDP.from_csr(S, A, torch.tensor(mdp["row_ptr"], device=dev), torch.tensor(mdp["col"], device=dev),
                            torch.tensor(val32, device=dev), torch.tensor(R32, device=dev), 0.9)
    V, V64, pi, st = m.value_iterate(tol=1e-8)
    assert st["certified"] == 1
    assert np.max(np.abs(V64.cpu().numpy() - Vo)) <= 1e-6 * max(1.0, np.max(np.abs(Vo)))
    bad, _ = policy_mismatches(pi.cpu().numpy(), pio, gapo)
    assert bad == 0


@pytest.mark.parametrize("fmt,padded", FORMS[1:])
def test_pipelined_csr_sweep_equals_direct_sweep(fmt, padded):
    """The shared-memory pipelined sweep and the direct-load sweep do the same arithmetic in
    the same order: their sweeps agree bitwise (values, policy, gap)."""
    native = native_or_skip()
    import torch

    p = MID
    mt = native.MDP.build(p, fmt=fmt, padded=padded)
    md = native.MDP.build(p, fmt=fmt, padded=padded, direct=True)
    g = torch.Generator(device="cuda").manual_seed(3)
    V = torch.rand(mt.S, device="cuda", generator=g) * 100
    outs = []
    for m in (mt, md):
        Vo = torch.empty_like(V)
        pi = torch.empty(m.S, dtype=torch.int32, device="cuda")
        gap = torch.empty_like(V)
        m.bellman32(V, Vo, pi, gap)
        torch.cuda.synchronize()
        outs.append((Vo, pi, gap))
    assert torch.equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][1], outs[1][1])
    assert torch.equal(outs[0][2], outs[1][2])
    # every schedule the autotuner may pick computes the same sweep
    us = mt.autotune(reps=3)
    assert us > 0
    Vo = torch.empty_like(V)
    mt.bellman32(V, Vo)
    torch.cuda.synchronize()
    assert torch.equal(Vo, outs[0][0])


@pytest.mark.parametrize("H", [9, 12])
def test_more_than_eight_hosts(H):
    """Instances with H > 8 run the kernels instantiated for 16 hosts (every H <= 8 has its
    own instantiation): implicit, CSR and sliced handles and a batch mixing H = 3 and H
    agree with the oracle's optimum within 1e-6 relative."""
    native = native_or_skip()
    p = inputs.make_params(H, 1, 1, 0.9, seed=11)
    Vs, pis, gaps, _ = oracle.solve(p, tol=1e-12)
    for kw in (dict(fmt="implicit"), dict(fmt="csr_f32"), dict(fmt="csr_f32", sliced=True)):
        m = native.MDP.build(p, **kw)
        _, V64, pi, st = m.value_iterate(tol=1e-6)
        assert st["certified"] == 1, kw
        assert rel_err(V64.cpu().numpy(), Vs) <= 1e-6, kw
        assert policy_mismatches(pi.cpu().numpy(), pis, gaps)[0] == 0, kw
        m.close()
    q = inputs.make_params(3, 2, 3, 0.95, seed=4)
    b = native.Batch([q, p])
    _, V64, pi, stats, rc = b.value_iterate(tol=1e-6)
    assert rc == native.VC_OK and all(s["certified"] == 1 for s in stats)
    off = b.offsets
    assert rel_err(V64.cpu().numpy()[off[1]:off[2]], Vs) <= 1e-6
    assert rel_err(V64.cpu().numpy()[off[0]:off[1]], oracle.solve(q, tol=1e-12)[0]) <= 1e-6
    b.close()
