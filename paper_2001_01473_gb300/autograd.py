"""torch.autograd.Function around the 2D FP32 sweep and its adjoint.

stencil_sweep(u0, coeffs, T, shape, radius) returns u_T = S^T(u0) computed by
the library; its backward calls the library's adjoint entry point
(an5d_run_adjoint), which returns dL/du0 on the interior (zero on the halo:
the halo is boundary data, not a parameter) and dL/dcoeffs.
"""
from __future__ import annotations

import numpy as np
import torch

from . import an5d

_plans: dict = {}


def _plan(shape: int, radius: int, coeffs: np.ndarray, dims) -> an5d.Plan:
    key = (shape, radius, tuple(np.asarray(coeffs, np.float64).tolist()), tuple(dims))
    p = _plans.get(key)
    if p is None:
        p = an5d.Plan(2, shape, radius, coeffs, "f32", dims)
        _plans[key] = p
    return p


class StencilSweep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, coeffs, T, shape, radius):
        if u0.dtype != torch.float32 or not u0.is_cuda or u0.dim() != 2:
            raise ValueError("u0 must be a 2D float32 CUDA tensor (padded grid)")
        dims = (u0.shape[0] - 2 * radius, u0.shape[1] - 2 * radius)
        c = coeffs.detach().double().cpu().numpy()
        plan = _plan(shape, radius, c, dims)
        u0c = u0.contiguous()
        out = torch.empty_like(u0c)
        plan.run(u0c, out, int(T))
        ctx.save_for_backward(u0c)
        ctx.plan, ctx.T, ctx.n = plan, int(T), c.size
        ctx.cdtype, ctx.cdevice = coeffs.dtype, coeffs.device
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (u0,) = ctx.saved_tensors
        grad_u0 = torch.empty_like(u0)
        gc = an5d.an5d_run_adjoint(ctx.plan.handle, u0, grad_out.contiguous(), grad_u0, ctx.T)
        grad_c = torch.from_numpy(gc[: ctx.n].copy()).to(dtype=ctx.cdtype, device=ctx.cdevice)
        return grad_u0, grad_c, None, None, None


def stencil_sweep(u0: torch.Tensor, coeffs: torch.Tensor, T: int, shape: int, radius: int):
    """u_T of T steps of the 2D stencil (canonical coefficient order), differentiable
    with respect to u0 (interior) and coeffs."""
    return StencilSweep.apply(u0, coeffs, T, shape, radius)
