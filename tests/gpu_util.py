"""Helpers for the GPU tests: run the CUDA path through the C ABI and compare
with the CPU oracle."""
from __future__ import annotations

import numpy as np

TOL_F32 = 2e-6      # relative L2 per transform, FP32 path


def rel_l2_rows(yr, yi, rr, ri) -> np.ndarray:
    """Relative L2 error of every row (both planes together)."""
    yr = np.asarray(yr, np.float64)
    yi = np.asarray(yi, np.float64)
    num = np.sum((yr - rr) ** 2 + (yi - ri) ** 2, axis=-1)
    den = np.sum(rr ** 2 + ri ** 2, axis=-1)
    return np.sqrt(num / np.where(den > 0, den, 1.0))


def gpu_run(xr: np.ndarray, xi: np.ndarray, direction: int = 0, plan=None, inplace=False):
    """Transform float32 planes on cuda:0 through the C ABI; returns numpy."""
    import torch

    from paper_2504_07264_gb300 import Plan
    batch, n = xr.shape
    own = plan is None
    if own:
        plan = Plan(n, batch)
    try:
        dxr = torch.from_numpy(np.ascontiguousarray(xr)).cuda()
        dxi = torch.from_numpy(np.ascontiguousarray(xi)).cuda()
        if inplace:
            yr, yi = plan.execute(direction, dxr, dxi, dxr, dxi)
        else:
            yr, yi = plan.execute(direction, dxr, dxi)
        torch.cuda.synchronize()
        return yr.cpu().numpy(), yi.cpu().numpy()
    finally:
        if own:
            plan.destroy()
