"""torch.autograd form of the Gaussian field (Eq. 3 of arxiv 2608.14112).

``gaussian_field(prims, shape)`` returns the field Vtilde of Eq. 3 at every
voxel centre as a differentiable function of the raw primitive records
(position, log-scales, quaternion, scalar, weight logit; Eq. 2).  Forward and
backward are the library's CUDA kernels (``gve_evaluate`` / ``gve_backward``):
nothing per pair or per voxel is saved between them -- the backward
recomputes the field per brick from the records -- so a 1024^3 field costs
no more memory in training than the field itself.

The gradient of the truncated field treats the truncation set as fixed (the
kept pairs at the current parameters), which is what the brick kernels and the
paper's closed-form engine compute.
"""
from __future__ import annotations

import torch

from . import gve


class GaussianFieldFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, prims: torch.Tensor, shape, opts):
        prims = prims.contiguous()
        out = gve.gve_evaluate(prims, shape, opts)
        ctx.save_for_backward(prims)
        ctx.opts = opts
        return out

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (prims,) = ctx.saved_tensors
        grad = gve.gve_backward(prims, grad_out.contiguous().float(), ctx.opts)
        return grad, None, None


def gaussian_field(prims: torch.Tensor, shape, opts: gve.EvalOptions | None = None) -> torch.Tensor:
    """Differentiable Eq. 3 field of shape ``(nz, ny, nx)``."""
    return GaussianFieldFn.apply(prims, tuple(int(s) for s in shape), opts or gve.EvalOptions())
