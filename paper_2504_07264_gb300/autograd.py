"""torch.autograd.Function over planar (re, im) tensors.

The forward map is the DFT of Eq. (1) on stacked real planes, [yr; yi] =
E_2N [xr; xi] (Eq. (5)); it is linear, so the gradient of any real loss is
E_2N^T applied to the output gradient -- the adjoint transform, which runs as
its own CUDA kernel.  Nothing is saved for backward except the plan.
"""
from __future__ import annotations

import threading

import torch

from .sdft import SDFT_F32, Plan

_cache_lock = threading.Lock()
_plans: dict[tuple, Plan] = {}


def get_plan(n: int, batch: int, device: torch.device, dtype: int = SDFT_F32) -> Plan:
    """A cached plan for (n, batch) on ``device`` and the current stream.

    A plan's device-side state (its status word; on the work-queue and
    two-pass schedules of long transforms, a work counter or a scratch area)
    is shared by every call on it, so calls that overlap on the GPU must not
    share a plan.  The cache is therefore keyed on the current CUDA stream as
    well: work issued from different streams gets different plans, and calls
    on one stream are ordered by that stream.
    """
    stream = torch.cuda.current_stream(device).cuda_stream
    key = (int(n), int(batch), int(dtype), device.index, int(stream))
    with _cache_lock:
        p = _plans.get(key)
        if p is None:
            with torch.cuda.device(device):
                p = Plan(n, batch, dtype)
            _plans[key] = p
        return p


def clear_plan_cache() -> None:
    with _cache_lock:
        for p in _plans.values():
            p.destroy()
        _plans.clear()


class SplitDFT(torch.autograd.Function):
    """(xr, xi) -> (yr, yi), forward DFT per row; backward = adjoint DFT."""

    @staticmethod
    def forward(ctx, xr: torch.Tensor, xi: torch.Tensor):
        if xr.shape != xi.shape or xr.dim() < 1:
            raise ValueError("xr and xi must have the same shape (..., N)")
        n = xr.shape[-1]
        batch = xr.numel() // n
        plan = get_plan(n, batch, xr.device)
        xr_c, xi_c = xr.contiguous(), xi.contiguous()
        yr, yi = plan.forward(xr_c, xi_c)
        ctx.plan = plan
        return yr, yi

    @staticmethod
    def backward(ctx, gr: torch.Tensor, gi: torch.Tensor):
        plan = ctx.plan
        if gr is None:
            gr = torch.zeros_like(gi)
        if gi is None:
            gi = torch.zeros_like(gr)
        dxr, dxi = plan.adjoint(gr.contiguous(), gi.contiguous())
        return dxr, dxi


class SplitDFTAdjoint(torch.autograd.Function):
    """(xr, xi) -> adjoint DFT per row; backward = forward DFT."""

    @staticmethod
    def forward(ctx, xr: torch.Tensor, xi: torch.Tensor):
        n = xr.shape[-1]
        plan = get_plan(n, xr.numel() // n, xr.device)
        ctx.plan = plan
        return plan.adjoint(xr.contiguous(), xi.contiguous())

    @staticmethod
    def backward(ctx, gr, gi):
        if gr is None:
            gr = torch.zeros_like(gi)
        if gi is None:
            gi = torch.zeros_like(gr)
        return ctx.plan.forward(gr.contiguous(), gi.contiguous())


def split_dft(xr: torch.Tensor, xi: torch.Tensor):
    """Differentiable forward DFT of every row of planar (xr, xi)."""
    return SplitDFT.apply(xr, xi)


def split_dft_adjoint(xr: torch.Tensor, xi: torch.Tensor):
    """Differentiable adjoint (unnormalised inverse) DFT of every row."""
    return SplitDFTAdjoint.apply(xr, xi)
