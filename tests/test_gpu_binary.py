"""The paper's binary-action model (A = {-1, 1}, Section V-B..V-E) built on the device
(vc_build_binary_mdp) against the FP64 oracle's own construction of it (pinned in
test_oracle_binary.py).

* CSR structure: row offsets and columns bit-exact; FP32 values within one FP32 rounding
  of the oracle's FP64 probabilities; BF16 bit patterns and row scales equal to the
  oracle's nearest-even renormalised form; rewards within one FP32 rounding.
* Solves (FP32 and BF16 storage, CSR and sliced sweeps, Eq. 18's backup and the
  self-transition solve), certifying the error: V64 within 1e-6 of the oracle's optimum of
  the exact model relative to max(|V*|, 1) (this model's values cross zero; the handle
  keeps the exact FP64 rows for its refinement), policy equal wherever the oracle's Q-gap
  exceeds 1e-6; the FP32 iterate of an FP32 handle within the
  FP32 bound of the oracle's optimum of the FP32-rounded matrix.
* Full size (2,235,331 states): the oracle's backup of EVERY state of the certified V64 is
  within gamma 1e-6 of it and its argmax equals the returned policy where the gap
  exceeds 1e-6.
* Errors: bad parameters, unsupported formats, gradient and greedy requests.
"""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

from gpu_common import native_or_skip, policy_mismatches

pytestmark = pytest.mark.gpu

_ref = {}


def _oracle(name):
    if name not in _ref:
        p = inputs.binary_workload(name)
        _ref[name] = (p, oracle.bin_build_csr(p), oracle.bin_solve(p, tol=1e-12))
    return _ref[name]


@pytest.mark.parametrize("fmt", ["csr_f32", "csr_bf16"])
@pytest.mark.parametrize("name", ["binary_tiny", "binary_mid"])
def test_binary_csr_structure_matches_oracle(name, fmt):
    native = native_or_skip()
    p, (rp, col, val, R), _ = _oracle(name)
    m = native.MDP.build_binary(p, fmt=fmt)
    info = m.info()
    S = oracle.bin_num_states(p)
    assert info["S"] == S and info["A"] == 2
    assert info["nnz_logical"] == len(col) and info["feasible_rows"] == int(np.isfinite(R).sum())
    g_rp, g_col, g_val, g_scale, g_R = (t.cpu().numpy() if t is not None else None for t in m.export_csr())
    assert np.array_equal(g_rp, rp) and np.array_equal(g_col, col)
    feas = np.isfinite(R)
    assert np.array_equal(np.isfinite(g_R), feas)
    assert np.all(np.abs(g_R[feas] - R[feas]) <= np.abs(R[feas]) * 2.0**-24 + 1e-30)
    if fmt == "csr_f32":
        assert np.all(np.abs(g_val.astype(np.float64) - val) <= np.spacing(val.astype(np.float32)))
    else:
        bits, _, scale = oracle.bf16_renormalised(rp, val, 2 * S)
        assert np.array_equal(g_val.view(np.uint16), bits)
        assert np.array_equal(g_scale[feas], scale[feas])
    m.close()


@pytest.mark.parametrize("kw", [dict(fmt="csr_f32"), dict(fmt="csr_bf16"), dict(fmt="csr_f32", sliced=True),
                                dict(fmt="csr_bf16", sliced=True), dict(fmt="csr_f32", direct=True)])
@pytest.mark.parametrize("name", ["binary_tiny", "binary_mid"])
def test_binary_solve_matches_oracle(name, kw):
    native = native_or_skip()
    p, (rp, col, val, R), (Vs, pis, gaps, _) = _oracle(name)
    m = native.MDP.build_binary(p, **kw)
    if kw.get("sliced"):
        assert m.info()["csr_sliced"] == 1 and m.info()["nnz_sliced"] > 0
    scale = np.maximum(np.abs(Vs), 1.0)
    for sl in (False, True):
        # values of this model cross zero, so the 1e-6 is taken relative to max(|V*|, 1),
        # and the error (not only the residual) is certified: |V64 - V*| <= tol / 2
        V, V64, pi, st = m.value_iterate(tol=1e-6, self_loop=sl, accurate=True)
        assert st["certified"] == 1 and st["residual64"] < 1e-6
        assert np.max(np.abs(V64.cpu().numpy() - Vs) / scale) <= 1e-6, (kw, sl)
        bad, n = policy_mismatches(pi.cpu().numpy(), pis, gaps)
        assert bad == 0 and n > 0, (kw, sl)
    if kw["fmt"] == "csr_f32" and not kw.get("sliced") and not kw.get("direct"):
        # the FP32 iterate solves the FP32-rounded matrix: within the FP32 bound of its optimum
        S = len(Vs)
        v32 = val.astype(np.float32).astype(np.float64)
        V32o, _ = oracle.vi_csr(S, 2, rp, col, v32, R.astype(np.float32).astype(np.float64), p["gamma"], tol=1e-12)
        V, _, _, st = m.value_iterate(tol=1e-6, fp32_only=True)
        gam = p["gamma"]
        vmax = np.abs(V32o).max()
        ulp = float(np.spacing(np.float32(vmax)))
        bound = gam / (1 - gam) * st["residual"] + 2 * ulp / (1 - gam) + gam * 2.0**-24 * vmax / (1 - gam)
        assert np.max(np.abs(V.cpu().numpy().astype(np.float64) - V32o)) <= bound
    m.close()


def test_binary_full_size_every_state():
    native = native_or_skip()
    p = inputs.binary_workload("binary")
    S = oracle.bin_num_states(p)
    m = native.MDP.build_binary(p, fmt="csr_f32", sliced=True)
    m.autotune(reps=3)
    info = m.info()
    assert info["S"] == S == 2_235_331 and info["nnz_logical"] == 107_096_605
    _, V64, pi, st = m.value_iterate(tol=1e-6)
    assert st["certified"] == 1 and st["residual64"] < 1e-6
    V64 = V64.cpu().numpy()
    Tv, pio, gapo = oracle.bin_backup_all(p, V64)
    assert float(np.max(np.abs(Tv - V64))) <= p["gamma"] * 1e-6 + 1e-9
    sel = gapo > 1e-6
    assert int(np.sum(pi.cpu().numpy()[sel] != pio[sel])) == 0
    assert int(sel.sum()) > S // 2
    m.close()


def test_binary_errors():
    native = native_or_skip()
    import torch

    p = inputs.binary_workload("binary_tiny")
    for key, bad in (("J", 0), ("J", 9), ("H", 0), ("H", 17), ("C", 0), ("gamma", 1.0), ("lam", 0.0)):
        q = dict(p)
        q[key] = bad
        if key == "H" and bad > 0:
            q["mu"] = [0.5] * bad
            q["delta"] = [0.05] * bad
        with pytest.raises(native.VcError) as e:
            native.MDP.build_binary(q)
        assert e.value.code == native.VC_ERR_ARG, key
    q = dict(p)
    q["mu"] = [0.5, -1.0]
    with pytest.raises(native.VcError):
        native.MDP.build_binary(q)
    with pytest.raises(native.VcError):
        native.MDP.build_binary(p, fmt="implicit")
    m = native.MDP.build_binary(p)
    with pytest.raises(native.VcError) as e:
        m.greedy_policy()
    assert e.value.code == native.VC_ERR_ARG
    S = m.S
    V = torch.zeros(S, dtype=torch.float64, device="cuda")
    with pytest.raises(native.VcError) as e:
        m.value_grad(V, torch.zeros(S, dtype=torch.int32, device="cuda"), V + 1.0 / S)
    assert e.value.code == native.VC_ERR_ARG
    m.close()
