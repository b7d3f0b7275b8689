"""Split-precision tensor-core path (GPU): SDFT_F32_SPLIT_BF16 / _FP16.

Radix-R blocks of Eq. (5) run as tcgen05 GEMMs on hi/lo 16-bit splits with
float32 accumulation (N = 256 and 1024).  The paper states no precision; the
bound is the one set for this path: relative L2 error <= 1e-5 against the
float64 oracle over the batch, with the worst single transform reported.
Inputs: magnitudes 10^U(-3,3) with uniform phase (seed 3).
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import rel_l2_rows
from oracle import oracle as O

pytestmark = pytest.mark.gpu
TOL_SPLIT = 1e-5
DTYPES = {"bf16": 1, "fp16": 2}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_2504_07264_gb300 import build
    build.build()
    O.build()


def _run(xr, xi, dtype, direction=0, grid=None):
    import torch

    from paper_2504_07264_gb300 import Plan
    batch, n = xr.shape
    with Plan(n, batch, dtype) as plan:
        if grid is not None:
            plan.set_grid(grid)
            assert plan.grid == grid
        yr, yi = plan.execute(direction, torch.from_numpy(xr).cuda(), torch.from_numpy(xi).cuda())
        torch.cuda.synchronize()
        status = plan.sync_status()
    assert status == 0
    return yr.cpu().numpy(), yi.cpu().numpy()


def _global_rel(yr, yi, rr, ri):
    num = np.sum((yr - rr) ** 2 + (yi - ri) ** 2)
    return float(np.sqrt(num / np.sum(rr ** 2 + ri ** 2)))


@pytest.mark.parametrize("n", [256, 1024])
@pytest.mark.parametrize("dt", sorted(DTYPES))
@pytest.mark.parametrize("direction", [0, 1])
def test_split_matches_oracle(n, dt, direction):
    batch = 2 * (128 * 128 // n) // 16 + 9          # several tiles and a ragged tail
    xr, xi = W.logmag_phase_planes(n, batch, seed=3)
    yr, yi = _run(xr, xi, DTYPES[dt], direction)
    fn = O.dft_factored_dit if direction == 0 else O.adjoint_factored
    rr, ri = fn(xr, xi)
    g = _global_rel(yr, yi, rr, ri)
    worst = rel_l2_rows(yr, yi, rr, ri).max()
    assert g <= TOL_SPLIT, f"{dt} N={n}: global rel L2 {g:.3e} (worst transform {worst:.3e})"


@pytest.mark.parametrize("n", [256, 1024])
@pytest.mark.parametrize("dt", sorted(DTYPES))
@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("grid", [1, 4])
def test_split_several_tiles_per_cta(n, dt, direction, grid):
    """A small grid, so that every CTA runs at least three tiles of 128 GEMM
    rows (128/R transforms each) and the last tile is partial: the persistent
    tile loop -- operand-region reuse after the output copy, the next tile's
    prefetch, the mbarrier phases carried from tile to tile -- against the
    float64 oracle, transform by transform."""
    tpt = 128 // int(round(n ** 0.5))              # transforms per tile (R = sqrt(N))
    batch = 3 * grid * tpt + 1
    xr, xi = W.logmag_phase_planes(n, batch, seed=30 + n % 7 + 2 * direction + grid)
    yr, yi = _run(xr, xi, DTYPES[dt], direction, grid=grid)
    fn = O.dft_factored_dit if direction == 0 else O.adjoint_factored
    rr, ri = fn(xr, xi)
    g = _global_rel(yr, yi, rr, ri)
    rows = rel_l2_rows(yr, yi, rr, ri)
    worst = int(np.argmax(rows))
    assert np.isfinite(yr).all() and np.isfinite(yi).all()
    assert g <= TOL_SPLIT, (f"{dt} N={n} grid {grid}: global rel L2 {g:.3e} "
                            f"(worst transform {worst}: {rows[worst]:.3e})")
    # every transform, the partial last tile's included, carries the bound too
    assert rows.max() <= 4 * TOL_SPLIT, f"transform {worst}: {rows[worst]:.3e}"


@pytest.mark.parametrize("dt", sorted(DTYPES))
@pytest.mark.parametrize("direction", [0, 1])
def test_split_full_size_bandwidth_config(dt, direction):
    """N = 1024, batch 65536 (iid N(0,1), seed 1): the benchmark's split
    plan and grid.  128 sampled transforms against the float64 oracle,
    Parseval (forward) or its adjoint form on every transform."""
    import torch

    from paper_2504_07264_gb300 import Plan
    xr, xi = W.bandwidth()
    n, batch = W.BANDWIDTH["n"], W.BANDWIDTH["batch"]
    with Plan(n, batch, DTYPES[dt]) as plan:
        dxr = torch.from_numpy(xr).cuda()
        dxi = torch.from_numpy(xi).cuda()
        yr, yi = plan.execute(direction, dxr, dxi)
        e_in = (dxr.double() ** 2 + dxi.double() ** 2).sum(1) * n
        e_out = (yr.double() ** 2 + yi.double() ** 2).sum(1)
        parseval = ((e_out - e_in).abs() / e_in).max().item()
        idx = np.sort(np.random.default_rng(11 + direction).choice(batch, 128, replace=False))
        sel = torch.from_numpy(idx).cuda()
        gr = yr.index_select(0, sel).cpu().numpy()
        gi = yi.index_select(0, sel).cpu().numpy()
        assert plan.sync_status() == 0
    fn = O.dft_factored_dit if direction == 0 else O.adjoint_factored
    rr, ri = fn(xr[idx], xi[idx])
    rows = rel_l2_rows(gr, gi, rr, ri)
    g = _global_rel(gr, gi, rr, ri)
    assert g <= TOL_SPLIT, f"{dt}: global rel L2 {g:.3e} (worst transform {rows.max():.3e})"
    assert parseval < 1e-4


@pytest.mark.parametrize("dt", sorted(DTYPES))
def test_split_unit_vectors(dt):
    """Each basis input gives one column of E_2N: every tensor-core GEMM entry
    and the hi/lo bookkeeping are exercised in isolation."""
    n = 256
    eye = np.eye(2 * n, dtype=np.float32)
    xr = np.ascontiguousarray(eye[:, :n])
    xi = np.ascontiguousarray(eye[:, n:])
    yr, yi = _run(xr, xi, DTYPES[dt])
    rr, ri = O.dft_direct(xr, xi)
    assert _global_rel(yr, yi, rr, ri) <= TOL_SPLIT


@pytest.mark.parametrize("dt", sorted(DTYPES))
def test_precision_workload_sampled(dt):
    """262144 transforms of N = 256 (the precision workload): 256 sampled
    transforms against the oracle, Parseval on every transform."""
    import torch

    from paper_2504_07264_gb300 import Plan
    xr, xi = W.precision()
    n, batch = W.PRECISION["n"], W.PRECISION["batch"]
    with Plan(n, batch, DTYPES[dt]) as plan:
        dxr = torch.from_numpy(xr).cuda()
        dxi = torch.from_numpy(xi).cuda()
        yr, yi = plan.forward(dxr, dxi)
        e_in = (dxr.double() ** 2 + dxi.double() ** 2).sum(1) * n
        e_out = (yr.double() ** 2 + yi.double() ** 2).sum(1)
        parseval = ((e_out - e_in).abs() / e_in).max().item()
        idx = np.sort(np.random.default_rng(8).choice(batch, 256, replace=False))
        sel = torch.from_numpy(idx).cuda()
        gr = yr.index_select(0, sel).cpu().numpy()
        gi = yi.index_select(0, sel).cpu().numpy()
        assert plan.sync_status() == 0
    rr, ri = O.dft_factored_dit(xr[idx], xi[idx])
    assert _global_rel(gr, gi, rr, ri) <= TOL_SPLIT
    assert parseval < 1e-4


@pytest.mark.parametrize("n", [256, 1024])
@pytest.mark.parametrize("dt", sorted(DTYPES))
@pytest.mark.parametrize("direction", [0, 1])
def test_split_power_of_two_scaling_exact(n, dt, direction):
    """Scaling the input by 2^k scales the output by exactly 2^k, bit for bit:
    FP16's block exponent moves by k and leaves every rounding where it was;
    BF16 is split unscaled, and with its float32 exponent range every split,
    product and rotation is exact under a power-of-two scale (no value here
    leaves the normal range).  A wrong or missing unscale, or a BF16 split
    that depended on the magnitude, breaks the equality."""
    batch = 2 * (128 * 128 // n) // 16 + 9
    xr, xi = W.normal_planes(n, batch, seed=11)
    yr, yi = _run(xr, xi, DTYPES[dt], direction)
    for k in (40, -40):
        s = np.float32(2.0 ** k)
        zr, zi = _run(xr * s, xi * s, DTYPES[dt], direction)
        assert np.array_equal(zr, yr * s) and np.array_equal(zi, yi * s), (dt, k)


@pytest.mark.parametrize("n", [256, 1024])
@pytest.mark.parametrize("dt", sorted(DTYPES))
@pytest.mark.parametrize("batch", [1, 2, 3, 5, 9])
def test_split_fewer_transforms_than_a_tile(n, dt, batch):
    """Batches that leave the tile (128 / sqrt(N) transforms: 8 at N = 256,
    4 at N = 1024) partly empty, or give most CTAs nothing to do: the empty
    rows are computed on whatever the buffer holds and never stored."""
    xr, xi = W.logmag_phase_planes(n, batch, seed=30 + batch)
    for direction, fn in ((0, O.dft_factored_dit), (1, O.adjoint_factored)):
        yr, yi = _run(xr, xi, DTYPES[dt], direction)
        rr, ri = fn(xr, xi)
        assert _global_rel(yr, yi, rr, ri) <= TOL_SPLIT
        assert rel_l2_rows(yr, yi, rr, ri).max() <= 4 * TOL_SPLIT


@pytest.mark.parametrize("n", [256, 1024])
@pytest.mark.parametrize("dt", sorted(DTYPES))
def test_split_in_place(n, dt):
    """yr == xr and yi == xi, with several tiles per CTA (a small grid): a tile's
    outputs are written while later tiles' inputs are still to be read."""
    import torch

    from paper_2504_07264_gb300 import Plan
    tpt = 128 // int(round(n ** 0.5))
    grid = 4
    batch = 3 * grid * tpt + 1
    xr, xi = W.logmag_phase_planes(n, batch, seed=41)
    with Plan(n, batch, DTYPES[dt]) as plan:
        plan.set_grid(grid)
        dxr = torch.from_numpy(xr).cuda()
        dxi = torch.from_numpy(xi).cuda()
        plan.execute(0, dxr, dxi, dxr, dxi)             # forward in place
        torch.cuda.synchronize()
        yr, yi = dxr.cpu().numpy(), dxi.cpu().numpy()
        plan.execute(1, dxr, dxi, dxr, dxi)             # then the adjoint in place
        torch.cuda.synchronize()
        zr, zi = dxr.cpu().numpy(), dxi.cpu().numpy()
        assert plan.sync_status() == 0
    rr, ri = O.dft_factored_dit(xr, xi)
    assert _global_rel(yr, yi, rr, ri) <= TOL_SPLIT
    qr, qi = O.adjoint_factored(yr, yi)                 # of what the GPU wrote
    assert _global_rel(zr, zi, qr, qi) <= TOL_SPLIT
