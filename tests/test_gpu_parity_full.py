"""GPU parity at the full workload sizes (2.5 M and 12.5 M states), where the oracle
cannot run value iteration to the optimum in test time but can back up every state once:

* certificate: the oracle's own Bellman backup of the returned V64, over EVERY state
  (contiguous state ranges on all host cores), satisfies |T(V64)(s) - V64(s)| <=
  gamma * 1e-6 (one oracle Bellman step of a certified iterate), so by the contraction
  bound V64 is within gamma/(1-gamma) * 1e-6 of V* everywhere;
* the returned policy equals the oracle's argmax of T(V64) at every state whose oracle
  Q-gap exceeds 1e-6;
* the logical successor count equals the oracle's own count.
"""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

from gpu_common import native_or_skip

pytestmark = pytest.mark.gpu

CASES = [("large", "implicit", False, False), ("large", "csr_f32", False, False), ("large", "csr_f32", True, False),
         ("large", "csr_bf16", False, False), ("precision", "csr_bf16", True, False),
         ("precision", "implicit", False, False),
         # the sliced copy, autotuned as the benchmark runs it (the large padded case is the
         # benchmark's headline configuration)
         ("large", "csr_f32", True, True), ("large", "csr_bf16", True, True), ("precision", "csr_bf16", False, True),
         ("precision", "csr_f32", False, True)]


@pytest.mark.parametrize("name,fmt,padded,sliced", CASES)
def test_full_size_certificate_and_every_state_backup(name, fmt, padded, sliced):
    native = native_or_skip()
    p = inputs.workload(name)
    m = native.MDP.build(p, fmt=fmt, padded=padded, sliced=sliced)
    if sliced:
        m.autotune(reps=3)
        assert m.info()["csr_sliced"] == 1
    info = m.info()
    S = oracle.num_states(p)
    assert info["S"] == S
    if padded:
        assert info["nnz_stored"] == S * (p["H"] + 1) * (2 * p["H"] + 3)
    V, V64, pi, st = m.value_iterate(tol=1e-6)
    assert st["certified"] == 1 and st["residual64"] < 1e-6
    V64 = V64.cpu().numpy()
    pi = pi.cpu().numpy()
    Tv, pio, gapo = oracle.backup_all(p, V64)
    worst = float(np.max(np.abs(Tv - V64)))
    assert worst <= p["gamma"] * 1e-6 + 1e-9, worst
    sel = gapo > 1e-6
    bad = np.flatnonzero(sel & (pi != pio))
    assert bad.size == 0, (bad[:8], pi[bad[:8]], pio[bad[:8]], gapo[bad[:8]])
    assert int(sel.sum()) > S // 2
    m.close()


@pytest.mark.parametrize("name,nnz", [("large", 130_468_750), ("precision", 790_546_875), ("grad", 14_168_750)])
def test_logical_nnz_matches_closed_count(name, nnz):
    # canonical successor counts of the workloads, counted independently when they were
    # specified, and recounted by the oracle's own enumeration
    native = native_or_skip()
    p = inputs.workload(name)
    assert oracle.csr_nnz(p) == nnz
    m = native.MDP.build(p, fmt="implicit")
    assert m.info()["nnz_logical"] == nnz
    m.close()
    m2 = native.MDP.build(p, fmt="csr_f32")
    assert m2.info()["nnz_stored"] == nnz
    feasible = m2.info()["feasible_rows"]
    m2.close()
    # padded rows: fixed offsets, the fill itself tallies the logical entries
    m3 = native.MDP.build(p, fmt="csr_f32", padded=True)
    assert m3.info()["nnz_logical"] == nnz and m3.info()["feasible_rows"] == feasible
    m3.close()


def test_headline_configuration_equals_the_csr_kernel_bitwise():
    """The benchmark's headline (large padded matrix, sliced copy, autotuned) against the
    pipelined CSR kernel on the same matrix: one sweep from random values, and the whole
    FP32 iterate with its sweep count, are bitwise equal."""
    native = native_or_skip()
    import torch

    p = inputs.workload("large")
    ms = native.MDP.build(p, fmt="csr_f32", padded=True, sliced=True)
    ms.autotune(reps=3)
    assert ms.info()["csr_sliced"] == 1
    mc = native.MDP.build(p, fmt="csr_f32", padded=True)
    S = mc.S
    g = torch.Generator(device="cuda").manual_seed(1)
    V = torch.rand(S, device="cuda", generator=g) * 60
    outs = []
    for m in (ms, mc):
        Vo = torch.empty_like(V)
        pi = torch.empty(S, dtype=torch.int32, device="cuda")
        gap = torch.empty_like(V)
        m.bellman32(V, Vo, pi, gap)
        torch.cuda.synchronize()
        outs.append((Vo, pi, gap))
    for x, y in zip(*outs):
        assert torch.equal(x, y)
    V1, _, _, s1 = ms.value_iterate(tol=1e-6, fp32_only=True)
    V2, _, _, s2 = mc.value_iterate(tol=1e-6, fp32_only=True)
    assert s1["sweeps"] == s2["sweeps"] and torch.equal(V1, V2)
    ms.close()
    mc.close()
