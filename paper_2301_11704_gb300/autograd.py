"""J^2 of a curve as a differentiable PyTorch function.

J^2(u, lambda) = sum_m w_m |r_m|^2 (eq. cost_function_general with the
theta-trapezoid quadrature in s and the grid sum in x), r = f(u) - lambda D_t u
(eq. residual_definition), as a function of the interior sections' grid values
u[1..M] (the end sections u_+ and u_- are fixed).  The backward pass returns the
exact gradient of this discrete J^2: the adjoint of the discretised residual
(the s-term -lambda W^-1 D_t^T W r of eq. KSE_G's discrete counterpart),
-2 dx w_m G_m for u and -2 <D_t u, r>_W for lambda.

Nothing but the inputs is kept between forward and backward: the backward pass
loads u into the curve again and recomputes r and its spectra (recomputation
instead of stored spectra).
"""
from __future__ import annotations

import torch

from .curve import KSCurve


class KSCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u_interior: torch.Tensor, lam: torch.Tensor, curve: KSCurve, ends: torch.Tensor):
        full = torch.cat([ends[:1], u_interior.to(curve.dtype), ends[1:]], dim=0)
        curve.set_state(full, float(lam), 0.0)
        J2, _ = curve.cost()
        ctx.curve = curve
        ctx.save_for_backward(u_interior, lam, ends)
        return torch.tensor(J2, dtype=torch.float64, device=u_interior.device)

    @staticmethod
    def backward(ctx, grad_out):
        u_interior, lam, ends = ctx.saved_tensors
        curve = ctx.curve
        full = torch.cat([ends[:1], u_interior.to(curve.dtype), ends[1:]], dim=0)
        curve.set_state(full, float(lam), 0.0)
        g, dJdl = curve.gradient(euclidean=True)
        go = grad_out.to(torch.float64)
        gu = (g[1:-1].to(torch.float64) * go).to(u_interior.dtype) if ctx.needs_input_grad[0] else None
        gl = (go * dJdl).to(lam.dtype) if ctx.needs_input_grad[1] else None
        return gu, gl, None, None


class CurveCost(torch.nn.Module):
    """J^2 of a curve with fixed end sections u_plus (s -> +inf) and u_minus
    (s -> -inf), differentiable in the interior sections and in lambda.

        cost = CurveCost(L=22.0, nx=64, ns=1024, S=102.3, u_plus=up, u_minus=um)
        J2 = cost(u_interior, lam)      # u_interior: [ns - 2, nx]
        J2.backward()
    """

    def __init__(self, L: float, nx: int, ns: int, S: float, u_plus, u_minus, *, s0: float = 0.0,
                 precision: str = "fp64", device=None):
        super().__init__()
        self.curve = KSCurve(L, nx, ns, S, u_plus, u_minus, s0=s0, precision=precision, adjoint="discrete",
                             device=device)
        dev = self.curve.device
        self.register_buffer("ends", torch.stack([torch.as_tensor(u_plus, dtype=self.curve.dtype, device=dev),
                                                  torch.as_tensor(u_minus, dtype=self.curve.dtype, device=dev)]))

    def forward(self, u_interior: torch.Tensor, lam=None) -> torch.Tensor:
        if lam is None:
            lam = torch.tensor(1.0, dtype=torch.float64, device=u_interior.device)
        return KSCost.apply(u_interior, lam, self.curve, self.ends)
