"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP32 forward and adjoint at every N = 2 .. 65536 on seeded inputs spanning
several CTA tiles plus a ragged tail; the full-size N = 1024 x 65536 batch in
the benchmark's launch configuration on sampled transforms plus Parseval on
every transform; bit-exact integer bins; in-place calls; host-buffer calls;
the DFT's closed forms and identities (delta, constant, tone, Parseval,
linearity, F(F(x))); argument errors that need a device.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import TOL_F32, gpu_run, rel_l2_rows
from oracle import oracle as O

pytestmark = pytest.mark.gpu

LOGNS = list(range(1, 17))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2504_07264_gb300 import build
    build.build()
    O.build()


def _batch_for(n: int) -> int:
    # several tiles of every kernel plus a ragged tail
    return max(3, (1 << 17) // n) + 1


@pytest.mark.parametrize("logn", LOGNS)
def test_forward_matches_oracle(logn):
    n = 1 << logn
    xr, xi = W.normal_planes(n, _batch_for(n), seed=100 + logn)
    yr, yi = gpu_run(xr, xi, 0)
    rr, ri = O.dft_factored_dit(xr, xi)
    err = rel_l2_rows(yr, yi, rr, ri)
    assert err.max() <= TOL_F32, f"N={n}: max rel err {err.max():.3e}"


@pytest.mark.parametrize("logn", LOGNS)
def test_adjoint_matches_oracle(logn):
    n = 1 << logn
    xr, xi = W.normal_planes(n, _batch_for(n), seed=200 + logn)
    yr, yi = gpu_run(xr, xi, 1)
    rr, ri = O.adjoint_factored(xr, xi)
    err = rel_l2_rows(yr, yi, rr, ri)
    assert err.max() <= TOL_F32, f"N={n}: max rel err {err.max():.3e}"


@pytest.mark.parametrize("logn", [1, 4, 6, 10, 12, 16])
def test_direct_oracle_agrees(logn):
    """Against the O(N^2) definition as well (small batches)."""
    n = 1 << logn
    xr, xi = W.uniform_planes(n, 3 if n <= 4096 else 1, seed=300 + logn)
    yr, yi = gpu_run(xr, xi, 0)
    if n <= 4096:
        rr, ri = O.dft_direct(xr, xi)
        err = rel_l2_rows(yr, yi, rr, ri)
    else:
        bins = np.random.default_rng(7).choice(n, 64, replace=False)
        rr, ri = O.dft_direct_bins(xr, xi, bins)
        err = rel_l2_rows(yr[:, bins], yi[:, bins], rr, ri)
    assert err.max() <= TOL_F32


def test_plain_config_n16():
    """1024 transforms of N = 16, U[-1, 1) seed 0: against both oracles."""
    xr, xi = W.plain()
    yr, yi = gpu_run(xr, xi, 0)
    for ref in (O.dft_direct(xr, xi), O.dft_factored_dit(xr, xi)):
        assert rel_l2_rows(yr, yi, *ref).max() <= TOL_F32


@pytest.mark.parametrize("logn", range(1, 7))
def test_integer_inputs_bit_exact(logn):
    """Integer inputs, N <= 64: bins 0, N/4, N/2, 3N/4 (all bins for N <= 4)
    equal the float64 oracle rounded to float32, bit for bit."""
    n = 1 << logn
    xr, xi = W.integer_planes(n, 257)
    yr, yi = gpu_run(xr, xi, 0)
    rr, ri = O.dft_direct(xr, xi)
    bins = list(range(n)) if n <= 4 else [0, n // 4, n // 2, 3 * n // 4]
    er = rr[:, bins].astype(np.float32)
    ei = ri[:, bins].astype(np.float32)
    assert np.array_equal(yr[:, bins].view(np.uint32), er.view(np.uint32))
    assert np.array_equal(yi[:, bins].view(np.uint32), ei.view(np.uint32))
    assert rel_l2_rows(yr, yi, rr, ri).max() <= TOL_F32


@pytest.mark.parametrize("logn", [3, 10, 13, 16])
def test_in_place(logn):
    n = 1 << logn
    xr, xi = W.normal_planes(n, _batch_for(n), seed=400 + logn)
    a = gpu_run(xr, xi, 0)
    b = gpu_run(xr, xi, 0, inplace=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("logn", [4, 10, 12, 16])
def test_adjoint_identities(logn):
    """adjoint(forward(x)) = N x, and adjoint(xr, xi) = swap(forward(xi, xr))."""
    n = 1 << logn
    xr, xi = W.normal_planes(n, 9, seed=500 + logn)
    yr, yi = gpu_run(xr, xi, 0)
    zr, zi = gpu_run(yr, yi, 1)
    assert rel_l2_rows(zr, zi, n * xr.astype(np.float64), n * xi.astype(np.float64)).max() < 4e-6
    ar, ai = gpu_run(xr, xi, 1)
    sr, si = gpu_run(xi, xr, 0)
    assert rel_l2_rows(ar, ai, si.astype(np.float64), sr.astype(np.float64)).max() < 4e-6


def test_full_size_bandwidth_config():
    """N = 1024, batch 65536 (256 MiB per plane), iid N(0,1) seed 1, in the
    benchmark's plan: 128 sampled transforms against the oracle, Parseval on
    every transform."""
    import torch

    from paper_2504_07264_gb300 import Plan
    xr, xi = W.bandwidth()
    n, batch = 1024, 65536
    with Plan(n, batch) as plan:
        dxr = torch.from_numpy(xr).cuda()
        dxi = torch.from_numpy(xi).cuda()
        yr, yi = plan.forward(dxr, dxi)
        e_in = (dxr.double() ** 2 + dxi.double() ** 2).sum(1) * n
        e_out = (yr.double() ** 2 + yi.double() ** 2).sum(1)
        parseval = ((e_out - e_in).abs() / e_in).max().item()
        idx = np.sort(np.random.default_rng(1).choice(batch, 128, replace=False))
        sel = torch.from_numpy(idx).cuda()
        gr = yr.index_select(0, sel).cpu().numpy()
        gi = yi.index_select(0, sel).cpu().numpy()
    assert parseval < 1e-5
    rr, ri = O.dft_factored_dit(xr[idx], xi[idx])
    assert rel_l2_rows(gr, gi, rr, ri).max() <= TOL_F32


@pytest.mark.parametrize("logn", [5, 10, 12, 15, 16])
def test_host_buffers_match_device_path(logn):
    import torch

    from paper_2504_07264_gb300 import Plan
    from paper_2504_07264_gb300 import sdft as S
    n = 1 << logn
    batch = max(2, (1 << 21) // n) + 1
    xr, xi = W.normal_planes(n, batch, seed=600 + logn)
    with Plan(n, batch) as plan:
        dev = gpu_run(xr, xi, 0, plan=plan)
        hxr = torch.from_numpy(xr).pin_memory()
        hxi = torch.from_numpy(xi).pin_memory()
        for mode in (S.SDFT_HOST_AUTO, S.SDFT_HOST_STAGED, S.SDFT_HOST_ZERO_COPY):
            hyr = torch.full_like(hxr, float("nan")).pin_memory()
            hyi = torch.full_like(hxi, float("nan")).pin_memory()
            plan.set_host_mode(mode)
            plan.execute_host(0, hxr, hxi, hyr, hyi)
            assert np.array_equal(dev[0], hyr.numpy()) and np.array_equal(dev[1], hyi.numpy()), mode
        # zero copy needs page-locked buffers; pageable ones are refused
        with pytest.raises(S.SdftError):
            plan.execute_host(0, xr, xi, np.empty_like(xr), np.empty_like(xi))


def test_argument_errors_on_device():
    import torch

    from paper_2504_07264_gb300 import sdft as S
    n, batch = 256, 8
    with S.Plan(n, batch) as plan:
        a = torch.zeros(batch * n + 8, device="cuda")
        b = torch.zeros(batch * n + 8, device="cuda")
        h = plan.handle
        p, q = a.data_ptr(), b.data_ptr()
        st = torch.cuda.current_stream().cuda_stream
        assert S.sdft_forward(h, p + 4, q, p + 64, q, st) == S.SDFT_ERR_MISALIGNED
        assert S.sdft_forward(h, p, q, p + 16, q + 16, st) == S.SDFT_ERR_ALIAS   # shifted in place
        c = torch.zeros(2 * batch * n, device="cuda")
        r = c.data_ptr()
        assert S.sdft_forward(h, p, q, r, r + 16, st) == S.SDFT_ERR_ALIAS        # outputs overlap
        assert S.sdft_forward(h, 0, q, p, q, st) == S.SDFT_ERR_INVALID_ARG
        assert S.sdft_execute(h, 5, p, q, r, r + 4 * batch * n, st) == S.SDFT_ERR_INVALID_ARG
        assert S.sdft_forward(h, p, q, p, q, st) == S.SDFT_OK                    # in place
        torch.cuda.synchronize()
        assert plan.sync_status() == S.SDFT_OK


@pytest.mark.parametrize("logn", [1, 2, 5, 8, 10, 11, 13, 14, 15, 16])
def test_invariants_on_gpu(logn):
    """The closed forms and identities of the DFT, on the GPU path with its
    tuned schedule: delta -> ones, constant -> N delta, a tone -> N delta at
    its bin, Parseval, linearity, and F(F(x))[n] = N x[-n mod N]."""
    n = 1 << logn
    k0 = (3 * n) // 4 + (1 if n > 4 else 0)
    rows = []
    delta = np.zeros(n, np.float32)
    delta[0] = 1.0
    rows.append((delta, np.zeros(n, np.float32)))
    rows.append((np.full(n, 0.5, np.float32), np.full(n, -0.25, np.float32)))
    ang = 2.0 * np.pi * ((k0 * np.arange(n)) % n) / n
    rows.append((np.cos(ang).astype(np.float32), np.sin(ang).astype(np.float32)))
    xr = np.stack([r for r, _ in rows])
    xi = np.stack([i for _, i in rows])
    yr, yi = (v.astype(np.float64) for v in gpu_run(xr, xi, 0))
    tol = 4e-6 * n
    assert np.abs(yr[0] - 1.0).max() < tol and np.abs(yi[0]).max() < tol
    expect_r = np.zeros(n)
    expect_i = np.zeros(n)
    expect_r[0], expect_i[0] = 0.5 * n, -0.25 * n
    assert np.abs(yr[1] - expect_r).max() < tol and np.abs(yi[1] - expect_i).max() < tol
    expect_r = np.zeros(n)
    expect_r[k0 % n] = n
    assert np.abs(yr[2] - expect_r).max() < tol and np.abs(yi[2]).max() < tol
    # Parseval, linearity and F(F(x)) on random rows
    a_r, a_i = W.normal_planes(n, 4, seed=700 + logn)
    b_r, b_i = W.normal_planes(n, 4, seed=800 + logn)
    fa = [v.astype(np.float64) for v in gpu_run(a_r, a_i, 0)]
    fb = [v.astype(np.float64) for v in gpu_run(b_r, b_i, 0)]
    e_in = (a_r.astype(np.float64) ** 2 + a_i.astype(np.float64) ** 2).sum(1) * n
    e_out = (fa[0] ** 2 + fa[1] ** 2).sum(1)
    assert np.abs(e_out - e_in).max() <= 1e-5 * e_in.max()
    c_r = (2.0 * a_r - 3.0 * b_r).astype(np.float32)
    c_i = (2.0 * a_i - 3.0 * b_i).astype(np.float32)
    fc = [v.astype(np.float64) for v in gpu_run(c_r, c_i, 0)]
    assert rel_l2_rows(fc[0], fc[1], 2.0 * fa[0] - 3.0 * fb[0], 2.0 * fa[1] - 3.0 * fb[1]).max() < 4e-6
    ffr, ffi = (v.astype(np.float64) for v in gpu_run(*gpu_run(a_r, a_i, 0), 0))
    rev = (-np.arange(n)) % n
    assert rel_l2_rows(ffr, ffi, n * a_r[:, rev].astype(np.float64),
                       n * a_i[:, rev].astype(np.float64)).max() < 4e-6
