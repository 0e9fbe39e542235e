"""Batch instances solved whole in one thread block (vc_batch_set_small_instances): the
instance's iterate lives in shared memory and it is swept to its own step-3 test without a
kernel launch per sweep.  It runs the graph loop's arithmetic, so with the path on or off the
FP32 iterates and sweep counts are equal bit for bit (Eq. 18's backup and the
self-transition solve), the certified values too, and they match the oracle's optimum."""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

from gpu_common import native_or_skip, policy_mismatches

pytestmark = pytest.mark.gpu


def _mixed():
    ps = inputs.batch_params(512, seed=2)
    S = [inputs.num_states(p["H"], p["C"], p["Q"]) for p in ps]
    small = [p for p, n in zip(ps, S) if n <= 12000][:24]
    large = [p for p, n in zip(ps, S) if 12000 < n <= 80000][:6]
    return small + large


@pytest.mark.parametrize("self_loop", [False, True])
def test_small_instance_path_is_bitwise_the_graph_loop(self_loop):
    native = native_or_skip()
    import torch

    ps = _mixed()
    b = native.Batch(ps)
    info = b.small_instances()
    S = [inputs.num_states(p["H"], p["C"], p["Q"]) for p in ps]
    assert info["count"] == sum(n <= info["max_states"] for n in S) and info["count"] >= 24
    runs = {}
    for on in (True, False):
        b.set_small_instances(info["max_states"] if on else 0)
        assert b.small_instances()["count"] == (info["count"] if on else 0)
        V, _, _, st, _ = b.value_iterate(tol=1e-6, fp32_only=True, self_loop=self_loop)
        _, V64, pi, st64, rc = b.value_iterate(tol=1e-6, self_loop=self_loop)
        assert rc == native.VC_OK
        runs[on] = (V, [s["sweeps"] for s in st], V64, pi, st64)
    assert torch.equal(runs[True][0], runs[False][0])
    assert runs[True][1] == runs[False][1]
    assert torch.equal(runs[True][2], runs[False][2]) and torch.equal(runs[True][3], runs[False][3])
    off = b.offsets
    V64 = runs[True][2].cpu().numpy()
    pi = runs[True][3].cpu().numpy()
    for i in (0, 5, 23):
        p = ps[i]
        Vs, pis, gaps, _ = oracle.solve(p, tol=1e-12)
        sl = slice(off[i], off[i + 1])
        assert np.max(np.abs(V64[sl] - Vs) / np.abs(Vs)) <= 1e-6
        assert policy_mismatches(pi[sl], pis, gaps)[0] == 0
    with pytest.raises(native.VcError):
        b.set_small_instances(-1)
    b.close()


def test_small_instances_under_the_block_iteration():
    """With VC_ITER_BLOCK a small instance is one block (the whole instance) iterated by the
    self-transition sweeps to its test: its FP32 iterate equals the self-transition loop's."""
    native = native_or_skip()
    import torch

    ps = _mixed()[:24]
    b = native.Batch(ps)
    Va, _, _, sa, _ = b.value_iterate(tol=1e-6, fp32_only=True, block=True)
    Vb, _, _, sb, _ = b.value_iterate(tol=1e-6, fp32_only=True, self_loop=True)
    assert torch.equal(Va, Vb) and [s["sweeps"] for s in sa] == [s["sweeps"] for s in sb]
    b.close()
