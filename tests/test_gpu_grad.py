"""GPU adjoint gradient (vc_value_grad) against the FP64 oracle.

* tiny instance (640 states): with the oracle's V* and policy as inputs the device
  gradient equals the oracle's dense-solve adjoint gradient (pinned by finite differences
  and the Euler identity) to 1e-9 relative; end to end (the device's own certified V64 and
  policy) within 1e-5 normwise (V64 carries the 1e-6 certificate), and against oracle central finite differences (h = 1e-4,
  solves to 1e-12) where the optimal policy does not change inside +-h, within 1e-5;
* the gradient workload (343,750 states): the returned lam satisfies the oracle's push
  form of the adjoint equation lam = rho + gamma P_pi^T lam to 1e-9, the gradient equals
  the oracle's contraction of the same (V64, pi, lam) to 1e-9 relative, and the Euler
  identity J = sum_w w dJ/dw holds (V* is 1-homogeneous in the reward weights);
* torch.autograd through VCValueFn returns the same gradient.

Tolerances: lam is refined in FP64 to a residual of 1e-11 (relative error ~1e-10 after the
1/(1-gamma) amplification); the contraction is FP64; end to end the 1e-6 certificate of V64
dominates.
"""
import numpy as np
import pytest

import oracle
from paper_2012_12419_gb300 import inputs

from gpu_common import native_or_skip

pytestmark = pytest.mark.gpu


def rho_empty_hosts(p):
    S = oracle.num_states(p)
    rho = np.zeros(S)
    C1, Q1 = p["C"] + 1, p["Q"] + 1
    for s in range(S):
        if (s // 2) // Q1 == 0:  # every occupancy digit zero
            rho[s] = 1.0
    return rho / rho.sum()


def _dev(x, torch, dtype=None):
    return torch.tensor(np.asarray(x), device="cuda", dtype=dtype)


def test_gradient_matches_dense_adjoint_and_fd_on_tiny():
    native = native_or_skip()
    import torch

    p = inputs.workload("tiny")
    rho = rho_empty_hosts(p)
    assert int(np.count_nonzero(rho)) == 2 * (p["Q"] + 1)
    Vs, pis, gaps, _ = oracle.solve(p, tol=1e-12)
    g_ref = oracle.grad_dense(p, Vs, pis, rho)
    m = native.MDP.build(p, fmt="implicit")
    # oracle optimum as input: isolates the adjoint solve and contraction
    dJ, lam, gs = m.value_grad(_dev(Vs, torch, torch.float64), _dev(pis, torch, torch.int32),
                               _dev(rho, torch, torch.float64), want_lambda=True)
    dJ = dJ.cpu().numpy()
    assert gs["residual64"] < 1e-11
    assert np.max(np.abs(dJ - g_ref)) < 1e-9 * np.max(np.abs(g_ref))
    assert gs["J"] == pytest.approx(float(rho @ Vs), rel=1e-14)
    # end to end from the device's own certified solve
    _, V64, pi, st = m.value_iterate(tol=1e-6)
    dJ2, _, _ = m.value_grad(V64, pi, _dev(rho, torch, torch.float64))
    dJ2 = dJ2.cpu().numpy()
    # V64 is within gamma/(1-gamma) * 1e-6 of V*; the value differences it feeds carry that
    assert np.max(np.abs(dJ2 - g_ref)) < 1e-5 * np.max(np.abs(g_ref))
    # central finite differences of the oracle's optimum
    theta = oracle.theta_vector(p)
    h = 1e-4
    checked = 0
    for i in range(len(theta)):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        Vp, pip, _, _ = oracle.solve(oracle.with_theta(p, tp), tol=1e-12)
        Vm, pim, _, _ = oracle.solve(oracle.with_theta(p, tm), tol=1e-12)
        if not (np.array_equal(pip, pis) and np.array_equal(pim, pis)):
            continue
        fd = (rho @ Vp - rho @ Vm) / (2 * h)
        assert dJ2[i] == pytest.approx(fd, rel=1e-5, abs=1e-6)
        checked += 1
    assert checked >= len(theta) - 2


def test_gradient_workload_full_size():
    native = native_or_skip()
    import torch

    p = inputs.workload("grad")
    S = oracle.num_states(p)
    assert S == 343_750
    rho = rho_empty_hosts(p)
    assert int(np.count_nonzero(rho)) == 22
    m = native.MDP.build(p, fmt="implicit")
    _, V64, pi, st = m.value_iterate(tol=1e-6)
    assert st["certified"] == 1
    dJ, lam, gs = m.value_grad(V64, pi, _dev(rho, torch, torch.float64), want_lambda=True)
    dJ = dJ.cpu().numpy()
    lam = lam.cpu().numpy()
    V64 = V64.cpu().numpy()
    pi = pi.cpu().numpy()
    assert gs["nnz_transpose"] > S
    # adjoint equation, checked with the oracle's own transitions (push form)
    resid = lam - rho - p["gamma"] * oracle.adjoint_apply(p, pi, lam)
    assert np.max(np.abs(resid)) < 1e-9
    # contraction against the oracle's analytic derivatives of every row
    g_ref = oracle.grad_contract(p, V64, pi, lam)
    assert np.max(np.abs(dJ - g_ref)) < 1e-9 * np.max(np.abs(g_ref))
    assert gs["J"] == pytest.approx(float(rho @ V64), rel=1e-12)
    # Euler identity in the reward weights: sum_w w dJ/dw = lam . R_pi = rho . V_pi exactly,
    # so J from the certified iterate V64 agrees within gamma/(1-gamma) * 1e-6 ...
    H = p["H"]
    w = np.array([p["w_occ"], p["w_loss"], p["w_q"]])
    assert abs(gs["J"] - float(w @ dJ[2 * H + 2:2 * H + 5])) < p["gamma"] / (1 - p["gamma"]) * 1e-6
    # ... and to 1e-9 once pi is evaluated to 1e-12
    Vpi, _ = m.evaluate_policy(torch.tensor(pi, device="cuda"), V0=torch.tensor(V64, device="cuda"), tol=1e-12)
    dJe, _, gse = m.value_grad(Vpi, torch.tensor(pi, device="cuda"), _dev(rho, torch, torch.float64))
    dJe = dJe.cpu().numpy()
    assert gse["J"] == pytest.approx(float(w @ dJe[2 * H + 2:2 * H + 5]), rel=1e-9)


def test_autograd_function_returns_the_adjoint_gradient():
    native = native_or_skip()
    import torch

    from paper_2012_12419_gb300.autograd import VCValueFn, theta_of

    p = inputs.workload("tiny")
    rho = torch.tensor(rho_empty_hosts(p), dtype=torch.float64)
    theta = torch.tensor(theta_of(p), dtype=torch.float64, requires_grad=True)
    base = {k: p[k] for k in ("H", "C", "Q", "gamma")}
    J = VCValueFn.apply(theta, base, rho)
    J.backward()
    Vs, pis, _, _ = oracle.solve(p, tol=1e-12)
    g_ref = oracle.grad_dense(p, Vs, pis, rho.numpy())
    # the forward solve's certificate bounds |V64 - V*| by gamma/(1-gamma) * 1e-6 (rho sums to 1)
    assert abs(float(J.detach()) - float(rho.numpy() @ Vs)) < p["gamma"] / (1 - p["gamma"]) * 1e-6
    g = theta.grad.numpy()
    assert np.max(np.abs(g - g_ref)) < 1e-5 * np.max(np.abs(g_ref))


def test_objective_entry_point_and_no_grad_forward():
    """vc_objective: rho . V in FP64 on the device equals the host dot product to rounding
    and the J that vc_value_grad reports; with S not a multiple of the block and S = 1.
    A forward pass without a gradient runs no adjoint solve and returns the same J."""
    native = native_or_skip()
    import torch

    from paper_2012_12419_gb300.autograd import VCValueFn, theta_of

    g = np.random.default_rng(4)
    for S in (1, 1023, 1025, 343_750):
        V = g.normal(30, 10, S)
        rho = g.random(S)
        J = native.objective(torch.tensor(V, device="cuda"), torch.tensor(rho, device="cuda"))
        J2 = native.objective(torch.tensor(V, device="cuda"), torch.tensor(rho, device="cuda"))
        assert float(J) == pytest.approx(float(np.dot(rho, V)), rel=1e-13)
        assert torch.equal(J, J2)
    with pytest.raises(ValueError):
        native.objective(torch.zeros(3, device="cuda"), torch.zeros(3, device="cuda"))
    p = inputs.workload("tiny")
    m = native.MDP.build(p, fmt="implicit")
    _, V64, pi, _ = m.value_iterate(tol=1e-6)
    rho = torch.tensor(rho_empty_hosts(p), dtype=torch.float64, device="cuda")
    _, _, gs = m.value_grad(V64, pi, rho)
    assert float(native.objective(V64, rho)) == pytest.approx(gs["J"], rel=1e-13)
    m.close()
    theta = torch.tensor(theta_of(p), dtype=torch.float64)
    base = {k: p[k] for k in ("H", "C", "Q", "gamma")}
    n0 = native.kernel_launches()
    with torch.no_grad():
        J0 = VCValueFn.apply(theta, base, rho.cpu())
    n1 = native.kernel_launches()
    thg = theta.clone().requires_grad_(True)
    J1 = VCValueFn.apply(thg, base, rho.cpu())
    n2 = native.kernel_launches()
    assert float(J0) == float(J1.detach())
    assert n2 - n1 > n1 - n0  # the adjoint solve ran only when theta required a gradient


def test_gradient_rejects_explicit_handles_and_bad_policies():
    native = native_or_skip()
    import torch

    p = inputs.workload("tiny")
    m = native.MDP.build(p, fmt="implicit")
    V = torch.zeros(640, dtype=torch.float64, device="cuda")
    rho = torch.ones(640, dtype=torch.float64, device="cuda") / 640
    bad = torch.zeros(640, dtype=torch.int32, device="cuda")  # placement on a vehicle in CCHI: infeasible
    with pytest.raises(native.VcError) as e:
        m.value_grad(V, bad, rho)
    assert e.value.code == native.VC_ERR_ARG
    rp = torch.tensor([0, 1], dtype=torch.int64, device="cuda")
    u = native.MDP.from_csr(1, 1, rp, torch.zeros(1, dtype=torch.int32, device="cuda"),
                            torch.ones(1, device="cuda"), torch.ones(1, device="cuda"), 0.9)
    with pytest.raises(native.VcError):
        u.value_grad(V[:1], torch.zeros(1, dtype=torch.int32, device="cuda"), rho[:1])
