"""torch.autograd.Function around the 2D FP32 sweep and its adjoint.

stencil_sweep(u0, coeffs, T, shape, radius) returns u_T = S^T(u0) computed by
the library; its backward calls the library's adjoint entry point
(an5d_run_adjoint), which returns dL/du0 on the interior (zero on the halo:
the halo is boundary data, not a parameter) and dL/dcoeffs.

Plans are cached per (device, stencil shape, radius, grid extents), at most
MAX_PLANS of them (least recently used first out); a call with new
coefficients updates the cached plan's coefficients in place
(an5d_plan_set_coeffs), so a training loop that changes the coefficients
every step keeps one plan and its device buffers.
"""
from __future__ import annotations

from collections import OrderedDict

import numpy as np
import torch

from . import an5d

MAX_PLANS = 8
_plans: "OrderedDict[tuple, an5d.Plan]" = OrderedDict()


def _plan(device: int, shape: int, radius: int, dims) -> an5d.Plan:
    key = (device, shape, radius, tuple(dims))
    p = _plans.get(key)
    if p is None:
        n = an5d.an5d_coeff_count(2, shape, radius)
        p = an5d.Plan(2, shape, radius, np.zeros(n), "f32", dims)
        _plans[key] = p
        while len(_plans) > MAX_PLANS:
            _, old = _plans.popitem(last=False)
            old.close()
    _plans.move_to_end(key)
    return p


class StencilSweep(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, coeffs, T, shape, radius):
        if u0.dtype != torch.float32 or not u0.is_cuda or u0.dim() != 2:
            raise ValueError("u0 must be a 2D float32 CUDA tensor (padded grid)")
        dims = (u0.shape[0] - 2 * radius, u0.shape[1] - 2 * radius)
        c = coeffs.detach().double().cpu().numpy()
        with torch.cuda.device(u0.device):
            plan = _plan(u0.device.index, shape, radius, dims)
            plan.set_coeffs(c)
            u0c = u0.contiguous()
            out = torch.empty_like(u0c)
            plan.run(u0c, out, int(T))
        ctx.save_for_backward(u0c)
        ctx.key = (u0.device.index, shape, radius, dims)
        ctx.c, ctx.T, ctx.n = c, int(T), c.size
        ctx.cdtype, ctx.cdevice = coeffs.dtype, coeffs.device
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (u0,) = ctx.saved_tensors
        with torch.cuda.device(u0.device):
            plan = _plan(*ctx.key)
            plan.set_coeffs(ctx.c)  # another forward may have changed them since
            grad_u0 = torch.empty_like(u0)
            gc = an5d.an5d_run_adjoint(plan.handle, u0, grad_out.contiguous(), grad_u0, ctx.T)
        grad_c = torch.from_numpy(gc[: ctx.n].copy()).to(dtype=ctx.cdtype, device=ctx.cdevice)
        return grad_u0, grad_c, None, None, None


def stencil_sweep(u0: torch.Tensor, coeffs: torch.Tensor, T: int, shape: int, radius: int):
    """u_T of T steps of the 2D stencil (canonical coefficient order), differentiable
    with respect to u0 (interior) and coeffs."""
    return StencilSweep.apply(u0, coeffs, T, shape, radius)
