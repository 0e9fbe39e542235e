"""The no-allocation sweep entry point against the handle-based sweep.

vc_bellman32_noalloc serves callers that cannot call cudaMalloc (device memory held by
another allocator's pool, latency-bound loops that must not risk an allocation's
synchronisation, code running under another library's stream capture): it keeps its
scratch in a static device array instead.  Through the C ABI, two calls in a row with
different inputs must reproduce vc_bellman32 on a VC_IMPLICIT handle of the same model
bitwise (same kernels, same arithmetic), return max|V_out - V| as the residual (+infinity
when a difference is NaN), accept NULL for the optional outputs, reject models larger
than the static scratch, and, once called outside a capture, replay from a CUDA graph
captured around a call.  This file is collected last so that a run stopping
at the first failure has already run every other test.
"""
import ctypes

import pytest

from paper_2012_12419_gb300 import inputs

from gpu_common import native_or_skip

pytestmark = pytest.mark.gpu


def _call(native, p, V, V_out, pi, res):
    L = native.load()
    cp, keep = native._params(p)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else None)
    rc = L.vc_bellman32_noalloc(ctypes.byref(cp), ptr(V), ptr(V_out), ptr(pi), ptr(res),
                                ctypes.c_void_p(native.torch.cuda.current_stream().cuda_stream))
    del keep
    return rc


@pytest.mark.parametrize("name", ["tiny", "mid"])
def test_noalloc_sweep_matches_handle_sweep_twice(name):
    native = native_or_skip()
    import torch

    p = inputs.workload("tiny") if name == "tiny" else inputs.make_params(4, 4, 6, 0.95, seed=7)
    m = native.MDP.build(p, fmt="implicit")
    S = m.S
    g = torch.Generator(device="cuda").manual_seed(5)
    for call in range(2):
        V = torch.rand(S, device="cuda", generator=g) * (50 + 30 * call)
        V_out = torch.full((S,), float("nan"), device="cuda")
        pi = torch.full((S,), -1, dtype=torch.int32, device="cuda")
        res = torch.full((1,), -1.0, device="cuda")
        assert _call(native, p, V, V_out, pi, res) == native.VC_OK
        ref = torch.empty_like(V)
        ref_pi = torch.empty_like(pi)
        m.bellman32(V, ref, ref_pi)
        torch.cuda.synchronize()
        assert torch.equal(V_out, ref)
        assert torch.equal(pi, ref_pi)
        assert res.item() == (V_out - V).abs().max().item()
    m.close()


def test_noalloc_optional_outputs_and_nan_residual():
    """pi and residual are optional; a NaN in the input makes the residual +infinity
    rather than a finite number (a NaN difference never drops out of the maximum)."""
    native = native_or_skip()
    import torch

    p = inputs.workload("tiny")
    m = native.MDP.build(p, fmt="implicit")
    S = m.S
    V = torch.rand(S, device="cuda", generator=torch.Generator(device="cuda").manual_seed(9)) * 40
    ref = torch.empty_like(V)
    m.bellman32(V, ref)
    out = torch.full_like(V, float("nan"))
    assert _call(native, p, V, out, None, None) == native.VC_OK
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    Vn = V.clone()
    Vn[17] = float("nan")
    res = torch.zeros(1, device="cuda")
    assert _call(native, p, Vn, out, None, res) == native.VC_OK
    torch.cuda.synchronize()
    assert res.item() == float("inf")
    # the residual word is cleared on every call: a clean input gives a finite value again
    pi = torch.empty(S, dtype=torch.int32, device="cuda")
    assert _call(native, p, V, out, pi, res) == native.VC_OK
    torch.cuda.synchronize()
    assert res.item() == (out - V).abs().max().item()
    m.close()


def test_noalloc_rejects_models_beyond_its_scratch():
    native = native_or_skip()
    import torch

    p = inputs.workload("large")  # 2,500,000 states > 1,048,576
    V = torch.zeros(8, device="cuda")
    out = torch.zeros(8, device="cuda")
    pi = torch.zeros(8, dtype=torch.int32, device="cuda")
    res = torch.zeros(1, device="cuda")
    assert _call(native, p, V, out, pi, res) == native.VC_ERR_ARG
    with pytest.raises(native.VcError):
        native.bellman32_noalloc(p, V, out, pi, res)


def test_noalloc_call_replays_from_a_captured_graph():
    """Stream capture by another library: after one call on the device (which looks up the
    static scratch's addresses), a call captured into a CUDA graph replays as a plain call.
    Each replay on new values in the captured V equals the handle sweep bitwise, policy
    and residual included."""
    native = native_or_skip()
    import torch

    p = inputs.workload("tiny")
    m = native.MDP.build(p, fmt="implicit")
    S = m.S
    g = torch.Generator(device="cuda").manual_seed(11)
    V = torch.rand(S, device="cuda", generator=g) * 60
    V_out = torch.empty_like(V)
    pi = torch.empty(S, dtype=torch.int32, device="cuda")
    res = torch.empty(1, device="cuda")
    assert _call(native, p, V, V_out, pi, res) == native.VC_OK  # first call: outside any capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        rc = _call(native, p, V, V_out, pi, res)
    assert rc == native.VC_OK
    ref = torch.empty_like(V)
    ref_pi = torch.empty_like(pi)
    for k in range(2):
        V.copy_(torch.rand(S, device="cuda", generator=g) * (40 + 25 * k))
        V_out.fill_(float("nan"))
        pi.fill_(-1)
        res.fill_(-1.0)
        graph.replay()
        m.bellman32(V, ref, ref_pi)
        torch.cuda.synchronize()
        assert torch.equal(V_out, ref)
        assert torch.equal(pi, ref_pi)
        assert res.item() == (V_out - V).abs().max().item()
    del graph
    m.close()
