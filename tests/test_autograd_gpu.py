"""Differentiation through the planar DFT (GPU): SplitDFT's backward is the
adjoint kernel, E_2N^T of Eq. (5).

Loss L = sum(w_r * yr^2 + w_i * yi^2) with (yr, yi) = DFT(xr, xi), weights iid
U[0, 1) (seed 2).  The gradient is checked against float64 central finite
differences of the same loss evaluated by the CPU oracle (N = 64, batch 8:
the loss is quadratic, so central differences carry no truncation error, only
rounding ~1e-10), and at the full autograd workload (N = 4096, batch 16384)
on sampled transforms against the oracle's analytic gradient 2 E^T (w * y).

Tolerance: the GPU gradient is a float32 forward transform, a float32
elementwise product and a float32 adjoint transform, each within 2e-6
relative L2 of exact; 4e-6 bounds their sum.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import rel_l2_rows
from oracle import oracle as O

pytestmark = pytest.mark.gpu
TOL_GRAD = 4e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_2504_07264_gb300 import build
    build.build()
    O.build()


def _gpu_grad(xr, xi, wr, wi):
    import torch

    from paper_2504_07264_gb300 import split_dft
    txr = torch.from_numpy(xr).cuda().requires_grad_(True)
    txi = torch.from_numpy(xi).cuda().requires_grad_(True)
    twr = torch.from_numpy(wr).cuda()
    twi = torch.from_numpy(wi).cuda()
    yr, yi = split_dft(txr, txi)
    loss = (twr * yr ** 2 + twi * yi ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    return txr.grad.cpu().numpy(), txi.grad.cpu().numpy(), loss.item()


def _loss64(xr, xi, wr, wi):
    yr, yi = O.dft_direct(xr, xi)
    return float(np.sum(wr * yr ** 2 + wi * yi ** 2))


def test_gradient_vs_central_differences():
    n, batch = 64, 8
    xr, xi = W.normal_planes(n, batch, seed=1)
    wr, wi = W.loss_weights(n, batch, seed=2)
    gr, gi, loss = _gpu_grad(xr, xi, wr, wi)
    x0r, x0i = xr.astype(np.float64), xi.astype(np.float64)
    w_r, w_i = wr.astype(np.float64), wi.astype(np.float64)
    assert abs(loss - _loss64(x0r, x0i, w_r, w_i)) / abs(loss) < 1e-5
    h = 1e-3
    fd_r = np.zeros_like(x0r)
    fd_i = np.zeros_like(x0i)
    for b in range(batch):
        for t in range(n):
            for plane, fd in ((x0r, fd_r), (x0i, fd_i)):
                keep = plane[b, t]
                plane[b, t] = keep + h
                lp = _loss64(x0r, x0i, w_r, w_i)
                plane[b, t] = keep - h
                lm = _loss64(x0r, x0i, w_r, w_i)
                plane[b, t] = keep
                fd[b, t] = (lp - lm) / (2 * h)
    err = rel_l2_rows(gr, gi, fd_r, fd_i)
    assert err.max() <= TOL_GRAD, f"max rel err vs central differences {err.max():.3e}"
    # the same against the analytic gradient 2 E^T (w * y) in float64
    yr, yi = O.dft_direct(x0r, x0i)
    ar, ai = O.adjoint_direct(2 * w_r * yr, 2 * w_i * yi)
    assert rel_l2_rows(fd_r, fd_i, ar, ai).max() < 1e-8   # the FD reference itself
    assert rel_l2_rows(gr, gi, ar, ai).max() <= TOL_GRAD


def test_full_autograd_workload_sampled():
    """N = 4096, batch 16384, iid N(0,1) seed 1, weights seed 2."""
    import torch

    from paper_2504_07264_gb300 import split_dft
    n, batch = W.AUTOGRAD["n"], W.AUTOGRAD["batch"]
    xr, xi = W.normal_planes(n, batch, seed=W.AUTOGRAD["seed"])
    wr, wi = W.loss_weights(n, batch, seed=W.AUTOGRAD["weight_seed"])
    txr = torch.from_numpy(xr).cuda().requires_grad_(True)
    txi = torch.from_numpy(xi).cuda().requires_grad_(True)
    twr, twi = torch.from_numpy(wr).cuda(), torch.from_numpy(wi).cuda()
    yr, yi = split_dft(txr, txi)
    (twr * yr ** 2 + twi * yi ** 2).sum().backward()
    idx = np.sort(np.random.default_rng(3).choice(batch, 48, replace=False))
    sel = torch.from_numpy(idx).cuda()
    gr = txr.grad.index_select(0, sel).cpu().numpy()
    gi = txi.grad.index_select(0, sel).cpu().numpy()
    x0r, x0i = xr[idx].astype(np.float64), xi[idx].astype(np.float64)
    orr, ori = O.dft_factored_dit(x0r, x0i)
    ar, ai = O.adjoint_factored(2 * wr[idx] * orr, 2 * wi[idx] * ori)
    assert rel_l2_rows(gr, gi, ar, ai).max() <= TOL_GRAD


def test_adjoint_function_backward_is_forward():
    import torch

    from paper_2504_07264_gb300 import split_dft_adjoint
    n, batch = 256, 5
    xr, xi = W.normal_planes(n, batch, seed=9)
    txr = torch.from_numpy(xr).cuda().requires_grad_(True)
    txi = torch.from_numpy(xi).cuda().requires_grad_(True)
    ar, ai = split_dft_adjoint(txr, txi)
    (ar.sum() + 2 * ai.sum()).backward()
    # d/dx of <1, Re(F^H x)> + 2 <1, Im(F^H x)> = E (the forward) applied to (1, 2)
    ones = np.ones((batch, n))
    er, ei = O.dft_direct(ones, 2 * ones)
    assert rel_l2_rows(txr.grad.cpu().numpy(), txi.grad.cpu().numpy(), er, ei).max() < TOL_GRAD
