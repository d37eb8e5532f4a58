"""torch.autograd wrapper of the differentiable forward model.

``chi2_of_final_density(white, target, plan, a)`` runs the linear field,
2LPT and the KDK steps (keeping dx at every stage), paints the final
density and returns chi^2 = sum (delta - target)^2 / sigma^2 (the
likelihood term of the paper's Eq. 12).  Its backward pass is the
hand-written adjoint chain of libfpm: chi^2 gradient, paint transpose,
reverse KDK from the checkpoints, 2LPT transpose and linear-field
transpose, giving d chi^2 / d white.  Only argument marshalling happens
here; every step runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from .binding import Plan


# Force checkpoints (the forward's force mesh and tile buckets at every
# stage) spare the reverse pass a paint, a force and a sort per step; they
# are kept when they fit in the device memory that is free or held unused by
# torch's caching allocator, with this margin to spare.
FORCE_CKPT_MARGIN_BYTES = 8 << 30


def _force_checkpoints(plan: Plan, nstages: int, device):
    need = nstages * plan.force_ckpt_floats * 4
    free, _ = torch.cuda.mem_get_info(device)
    cached = torch.cuda.memory_reserved(device) - torch.cuda.memory_allocated(device)
    if need + FORCE_CKPT_MARGIN_BYTES > free + cached:
        return None
    return torch.empty(nstages, plan.force_ckpt_floats, device=device)


class _Chi2OfFinalDensity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, white, target, plan: Plan, a, sigma: float, order: int):
        a = np.asarray(a, dtype=np.float64)
        lin_k = plan.linear_field(white.contiguous())
        dx, p = plan.lpt(lin_k, float(a[0]), order)
        ckpt = torch.empty(len(a), 3, plan.N, device=white.device)
        fckpt = _force_checkpoints(plan, len(a), white.device)
        plan.kdk(dx, p, a, ckpt=ckpt, fckpt=fckpt)
        rho = plan.paint(dx)
        loss, g_rho = plan.chi2(rho, target.contiguous(), sigma)
        ctx.plan, ctx.a, ctx.order = plan, a, order
        ctx.has_fckpt = fckpt is not None
        ctx.save_for_backward(lin_k, ckpt, g_rho, fckpt if fckpt is not None else ckpt[:0])
        return torch.tensor(loss, dtype=torch.float64, device=white.device)

    @staticmethod
    def backward(ctx, grad_out):
        lin_k, ckpt, g_rho, fckpt = ctx.saved_tensors
        plan, a = ctx.plan, ctx.a
        g_dx = plan.paint_adj(ckpt[-1], g_rho)
        g_dx, g_p = plan.kdk_adj(ckpt, a, g_dx, fckpt=fckpt if ctx.has_fckpt else None)
        g_lin_k = plan.lpt_adj(lin_k, float(a[0]), g_dx, g_p, ctx.order)
        g_white = plan.linear_field_adj(g_lin_k)
        return g_white * grad_out.to(g_white.dtype), None, None, None, None, None


def chi2_of_final_density(white, target, plan: Plan, a, sigma: float = 1.0, order: int = 2):
    """chi^2 between the final CIC density contrast and `target`, differentiable
    with respect to the white noise `white` (float32[np, np, np] on the GPU)."""
    return _Chi2OfFinalDensity.apply(white, target, plan, a, sigma, order)
