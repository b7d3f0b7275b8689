"""The allocation-free entry point for long transforms (GPU).

sdft_execute_noalloc serves callers that cannot allocate device memory: it
runs the N = 32768 / 65536 kernel on scratch and twiddle tables held in
file-scope device arrays instead of plan-owned cudaMalloc memory.  Its results
must match the float64 oracle and the plan-based entry point (sdft_execute on
a plan running the same two-pass kernel), on two calls in a row (the second
call reuses the arrays the first one left behind), out of place and in place.
This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import TOL_F32, rel_l2_rows
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2504_07264_gb300 import build
    build.build()
    O.build()


def _oracle(direction, xr, xi):
    fn = O.dft_factored_dit if direction == 0 else O.adjoint_factored
    return fn(xr, xi)


# batches above the slot count (32 at N = 32768, 16 at N = 65536), so that the
# CTAs take transforms in turn and reuse their scratch slots
@pytest.mark.parametrize("n,batch", [(32768, 37), (65536, 19)])
@pytest.mark.parametrize("direction", [0, 1])
def test_noalloc_matches_oracle(n, batch, direction):
    """Two calls in a row through the C ABI against the float64 oracle and
    against the plan-based entry point on the same kernel; the second call runs
    on the scratch the first one left behind."""
    import torch

    from paper_2504_07264_gb300 import Plan
    from paper_2504_07264_gb300 import sdft as S
    xr, xi = W.normal_planes(n, batch, seed=700 + n % 97 + direction)
    ref_r, ref_i = _oracle(direction, xr, xi)
    dxr = torch.from_numpy(xr).cuda()
    dxi = torch.from_numpy(xi).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    # the existing entry point, sdft_execute, on a plan whose schedule is the
    # same two-pass CTA kernel (plan-owned scratch and tables)
    large = [i for i in range(S.sdft_schedule_count(n, 0))
             if "two passes per CTA" in S.sdft_schedule_describe(n, 0, i)]
    assert large, "no two-pass CTA schedule for this length"
    prev = S.sdft_schedule_selected(n, 0)
    try:
        assert S.sdft_schedule_select(n, 0, large[0]) == S.SDFT_OK
        with Plan(n, batch) as plan:
            pr, pi = plan.execute(direction, dxr, dxi)
            torch.cuda.synchronize()
            assert plan.sync_status() == S.SDFT_OK
        pr, pi = pr.cpu().numpy(), pi.cpu().numpy()
    finally:
        S.sdft_schedule_select(n, 0, prev)
    for call in range(2):
        yr = torch.full_like(dxr, float("nan"))
        yi = torch.full_like(dxi, float("nan"))
        st = S.sdft_execute_noalloc(n, batch, direction, dxr.data_ptr(), dxi.data_ptr(),
                                    yr.data_ptr(), yi.data_ptr(), stream)
        assert st == S.SDFT_OK, S.sdft_status_string(st)
        torch.cuda.synchronize()
        gr, gi = yr.cpu().numpy(), yi.cpu().numpy()
        err = rel_l2_rows(gr, gi, ref_r, ref_i)
        assert err.max() <= TOL_F32, f"call {call}: max rel err {err.max():.3e}"
        diff = rel_l2_rows(gr, gi, pr.astype(np.float64), pi.astype(np.float64))
        assert diff.max() <= TOL_F32, f"call {call}: differs from sdft_execute by {diff.max():.3e}"


@pytest.mark.parametrize("n,batch", [(32768, 37), (65536, 19)])
def test_noalloc_in_place(n, batch):
    """In place (yr == xr, yi == xi), forward then adjoint, each against the
    oracle; the second call transforms the first one's output in place."""
    import torch

    from paper_2504_07264_gb300 import sdft as S
    xr, xi = W.normal_planes(n, batch, seed=750 + n % 89)
    fr, fi = _oracle(0, xr, xi)
    dr = torch.from_numpy(xr).cuda()
    di = torch.from_numpy(xi).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    st = S.sdft_execute_noalloc(n, batch, 0, dr.data_ptr(), di.data_ptr(), dr.data_ptr(),
                                di.data_ptr(), stream)
    assert st == S.SDFT_OK, S.sdft_status_string(st)
    torch.cuda.synchronize()
    gr, gi = dr.cpu().numpy(), di.cpu().numpy()
    err = rel_l2_rows(gr, gi, fr, fi)
    assert err.max() <= TOL_F32, f"forward in place: max rel err {err.max():.3e}"
    # adjoint of the GPU's own forward result, in place, against the oracle's
    # adjoint of those same float32 values
    ar, ai = _oracle(1, gr, gi)
    st = S.sdft_execute_noalloc(n, batch, 1, dr.data_ptr(), di.data_ptr(), dr.data_ptr(),
                                di.data_ptr(), stream)
    assert st == S.SDFT_OK, S.sdft_status_string(st)
    torch.cuda.synchronize()
    err = rel_l2_rows(dr.cpu().numpy(), di.cpu().numpy(), ar, ai)
    assert err.max() <= TOL_F32, f"adjoint in place: max rel err {err.max():.3e}"


def test_noalloc_rejects_other_lengths():
    import torch

    from paper_2504_07264_gb300 import sdft as S
    a = torch.zeros(1 << 17, device="cuda")
    b = torch.zeros(1 << 17, device="cuda")
    p, q = a.data_ptr(), b.data_ptr()
    half = (1 << 16) * 4
    for n in (1024, 16384, 131072):
        assert S.sdft_execute_noalloc(n, 1, 0, p, q, p + half, q + half, 0) == \
            S.SDFT_ERR_UNSUPPORTED_N
    assert S.sdft_execute_noalloc(32768, 0, 0, p, q, p + half, q + half, 0) == \
        S.SDFT_ERR_INVALID_ARG
