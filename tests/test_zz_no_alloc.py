"""The allocation-free entry point for long transforms (GPU).

sdft_execute_noalloc serves callers that cannot allocate device memory: it
runs the N = 32768 / 65536 kernel on scratch and twiddle tables held in
file-scope device arrays instead of plan-owned cudaMalloc memory.  Its results
must match the plan-based entry point, on two calls in a row (the second call
reuses the arrays the first one left behind).  This file is collected last so
that a run stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest

import workloads as W
from gpu_util import TOL_F32, rel_l2_rows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2504_07264_gb300 import build
    build.build()


@pytest.mark.parametrize("n,batch", [(32768, 37), (65536, 19)])
@pytest.mark.parametrize("direction", [0, 1])
def test_noalloc_matches_plan_entry_point(n, batch, direction):
    import torch

    from paper_2504_07264_gb300 import Plan
    from paper_2504_07264_gb300 import sdft as S
    xr, xi = W.normal_planes(n, batch, seed=700 + n % 97 + direction)
    dxr = torch.from_numpy(xr).cuda()
    dxi = torch.from_numpy(xi).cuda()
    with Plan(n, batch) as plan:
        rr, ri = plan.execute(direction, dxr, dxi)
    ref_r = rr.cpu().numpy().astype(np.float64)
    ref_i = ri.cpu().numpy().astype(np.float64)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        yr = torch.full_like(dxr, float("nan"))
        yi = torch.full_like(dxi, float("nan"))
        st = S.sdft_execute_noalloc(n, batch, direction, dxr.data_ptr(), dxi.data_ptr(),
                                    yr.data_ptr(), yi.data_ptr(), stream)
        assert st == S.SDFT_OK, S.sdft_status_string(st)
        torch.cuda.synchronize()
        err = rel_l2_rows(yr.cpu().numpy(), yi.cpu().numpy(), ref_r, ref_i)
        assert err.max() <= TOL_F32, f"call {call}: max rel err {err.max():.3e}"


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
