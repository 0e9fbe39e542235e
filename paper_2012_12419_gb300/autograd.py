"""torch.autograd.Function over the library's solve and adjoint gradient.

``VCValueFn.apply(theta, base, rho)`` returns J = rho . V*(theta) for the vehicular-cloud
placement MDP with parameters theta = (lambda, mu_1..mu_H, delta_1..delta_H, f, w_occ,
w_loss, w_q) on top of the fixed sizes and discount in ``base``.  The forward pass solves
the instance (``vc_value_iterate``) and takes J from the library (``vc_objective``); when
theta requires a gradient it also runs the adjoint solve (``vc_value_grad``) right away,
so the instance's handle and its device memory are released before forward returns and
the graph keeps only the 2H+5 derivatives, which backward scales by the incoming
gradient.  Every step runs in the CUDA library; this module only packs parameters.
The derivative is that of V_pi at the optimal policy, i.e. of V* wherever the optimal
action is unique (V* is piecewise smooth in theta, with kinks where the optimal policy
changes).
"""
from __future__ import annotations

import torch

from . import native


def theta_names(H: int):
    return ["lam"] + [f"mu{k}" for k in range(H)] + [f"delta{k}" for k in range(H)] + ["f", "w_occ", "w_loss", "w_q"]


def theta_of(p: dict) -> list:
    H = int(p["H"])
    return [float(p["lam"])] + [float(v) for v in p["mu"][:H]] + [float(v) for v in p["delta"][:H]] + [
        float(p["f"]), float(p["w_occ"]), float(p["w_loss"]), float(p["w_q"])]


def params_with(base: dict, theta) -> dict:
    """base (H, C, Q, gamma) with the 2H+5 parameters of theta."""
    H = int(base["H"])
    t = [float(v) for v in theta]
    if len(t) != 2 * H + 5:
        raise ValueError(f"theta needs {2 * H + 5} entries")
    p = dict(base)
    p["lam"] = t[0]
    p["mu"] = t[1:1 + H]
    p["delta"] = t[1 + H:1 + 2 * H]
    p["f"], p["w_occ"], p["w_loss"], p["w_q"] = t[1 + 2 * H:5 + 2 * H]
    return p


class VCValueFn(torch.autograd.Function):
    """J(theta) = rho . V*(theta), differentiable in theta through the adjoint kernels."""

    @staticmethod
    def forward(ctx, theta, base, rho, fmt="implicit", tol=1e-6, grad_tol=1e-11):
        p = params_with(base, theta.detach().cpu().tolist())
        m = native.MDP.build(p, fmt=fmt)
        try:
            _, V64, pi, _ = m.value_iterate(tol=tol)
            rho_d = rho.detach().to(device=V64.device, dtype=torch.float64).contiguous()
            J = native.objective(V64, rho_d)[0]
            dJ = None
            if ctx.needs_input_grad[0]:
                dJ, _, _ = m.value_grad(V64, pi, rho_d, tol=grad_tol)
        finally:
            m.close()
        ctx.dJ = dJ
        ctx.theta_device, ctx.theta_dtype = theta.device, theta.dtype
        return J.to(device=theta.device, dtype=theta.dtype)

    @staticmethod
    def backward(ctx, gJ):
        g = gJ.to(torch.float64) * ctx.dJ.to(gJ.device)
        return g.to(device=ctx.theta_device, dtype=ctx.theta_dtype), None, None, None, None, None
