"""Differentiable FHT: forward = fht_forward, backward = fht_adjoint (the
exact transpose of the recursion, i.e. the back-projection)."""
from __future__ import annotations

import torch

from . import _capi as C
from .fht import PlanCache

_cache = PlanCache(capacity=256)


class FHTFunction(torch.autograd.Function):
    """y = FHT(x) for one 2-D float image on a CUDA device (packed quadrants)."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, quads: int, boundary: str, split: str):
        plan = _cache.get(x.shape[0], x.shape[1], x.dtype, quads, boundary, split, x.device.index)
        ctx.plan = plan
        return plan.forward(x.contiguous())

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        plan = ctx.plan
        gin = plan.adjoint(g.contiguous().to(plan.out_dtype))
        return gin, None, None, None


def fht(x: torch.Tensor, quads: int = C.FHT_QALL, boundary: str = "cyclic", split: str = "T") -> torch.Tensor:
    """Differentiable transform of a float32/float64 image (autograd through the adjoint kernels)."""
    if x.dtype not in (torch.float32, torch.float64):
        raise ValueError("the differentiable transform takes float32 or float64 images")
    return FHTFunction.apply(x, quads, boundary, split)


def adjoint(plan, g: torch.Tensor) -> torch.Tensor:
    return plan.adjoint(g)
