"""Every compiled schedule of every length matches the oracle (GPU), and the
autotuner picks one of them."""
import re

import numpy as np
import pytest

import workloads as W
from gpu_util import TOL_F32, gpu_run, rel_l2_rows
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_2504_07264_gb300 import build
    build.build()
    O.build()


def _cases():
    from paper_2504_07264_gb300 import build
    from paper_2504_07264_gb300 import sdft as S
    build.build()
    out = []
    for m in range(1, 17):
        for i in range(1, max(1, S.sdft_schedule_count(1 << m, 0))):
            out.append((m, i))
    return out


@pytest.mark.parametrize("logn,idx", _cases())
def test_schedule_matches_oracle(logn, idx):
    from paper_2504_07264_gb300 import Plan
    from paper_2504_07264_gb300 import sdft as S
    n = 1 << logn
    batch = max(3, (1 << 16) // n) + 1
    xr, xi = W.normal_planes(n, batch, seed=900 + logn + idx)
    prev = S.sdft_schedule_selected(n, 0)
    try:
        assert S.sdft_schedule_select(n, 0, idx) == S.SDFT_OK
        with Plan(n, batch) as plan:
            assert S.sdft_schedule_describe(n, 0, idx).split(";")[0] in plan.describe()
            for direction, fn in ((0, O.dft_factored_dit), (1, O.adjoint_factored)):
                yr, yi = gpu_run(xr, xi, direction, plan=plan)
                assert rel_l2_rows(yr, yi, *fn(xr, xi)).max() <= TOL_F32
    finally:
        S.sdft_schedule_select(n, 0, prev)


def test_autotune_picks_a_schedule():
    from paper_2504_07264_gb300 import autotune as A
    from paper_2504_07264_gb300 import sdft as S
    prev = S.sdft_schedule_selected(4096, 0)
    try:
        rec = A.tune_one(4096, points=1 << 22, reps=3)
        assert 0 <= rec["index"] < S.sdft_schedule_count(4096, 0)
        assert len(rec["ms"]) == S.sdft_schedule_count(4096, 0) and min(rec["ms"]) > 0
        assert rec["ms"][rec["index"]] <= min(rec["ms"]) / (1 - 0.011)
        assert S.sdft_schedule_selected(4096, 0) == rec["index"]
    finally:
        S.sdft_schedule_select(4096, 0, prev)


def _cluster_indices(n):
    from paper_2504_07264_gb300 import build
    from paper_2504_07264_gb300 import sdft as S
    build.build()
    return [i for i in range(S.sdft_schedule_count(n, 0))
            if "cluster of" in S.sdft_schedule_describe(n, 0, i)]


@pytest.mark.parametrize("logn,idx", [(m, i) for m in (13, 14, 15, 16) for i in _cluster_indices(1 << m)])
def test_cluster_kernel_persistent_loop(logn, idx):
    """The cluster kernels with more transforms than resident clusters: every
    cluster runs several transforms, and the last one is ragged against the
    grid.  All transforms are checked against the oracle, both directions,
    and the second direction runs in place."""
    from paper_2504_07264_gb300 import Plan
    from paper_2504_07264_gb300 import sdft as S
    n = 1 << logn
    prev = S.sdft_schedule_selected(n, 0)
    try:
        assert S.sdft_schedule_select(n, 0, idx) == S.SDFT_OK
        q = int(re.search(r"cluster of (\d+) CTAs", S.sdft_schedule_describe(n, 0, idx)).group(1))
        with Plan(n, 1) as probe:
            clusters = probe.grid // q
        batch = 2 * clusters + 3
        xr, xi = W.normal_planes(n, batch, seed=950 + logn)
        with Plan(n, batch) as plan:
            assert "cluster of" in plan.describe()
            yr, yi = gpu_run(xr, xi, 0, plan=plan)
            assert rel_l2_rows(yr, yi, *O.dft_factored_dit(xr, xi)).max() <= TOL_F32
            zr, zi = gpu_run(xr, xi, 1, plan=plan, inplace=True)
            assert rel_l2_rows(zr, zi, *O.adjoint_factored(xr, xi)).max() <= TOL_F32
            assert plan.sync_status() == S.SDFT_OK
    finally:
        S.sdft_schedule_select(n, 0, prev)


def _prefetch_indices(n):
    from paper_2504_07264_gb300 import build
    from paper_2504_07264_gb300 import sdft as S
    build.build()
    return [i for i in range(S.sdft_schedule_count(n, 0))
            if "prefetched" in S.sdft_schedule_describe(n, 0, i)
            or "whole lines" in S.sdft_schedule_describe(n, 0, i)]


@pytest.mark.parametrize("logn,idx", [(m, i) for m in range(1, 14) for i in _prefetch_indices(1 << m)])
def test_prefetch_kernel_persistent_loop(logn, idx):
    """The prefetching and line-moving row kernels with more tiles than CTAs
    (every CTA loops, prefetching while it computes) and a last tile with
    fewer transforms than the CTA holds; both directions against the oracle,
    the adjoint in place."""
    from paper_2504_07264_gb300 import Plan
    from paper_2504_07264_gb300 import sdft as S
    n = 1 << logn
    per = int(re.search(r"(\d+) transform\(s\)/CTA tile", S.sdft_schedule_describe(n, 0, idx)).group(1))
    prev = S.sdft_schedule_selected(n, 0)
    try:
        assert S.sdft_schedule_select(n, 0, idx) == S.SDFT_OK
        with Plan(n, 1) as probe:
            grid = probe.grid
        batch = 2 * grid * per + max(1, per // 2) + 1
        xr, xi = W.normal_planes(n, batch, seed=960 + logn)
        with Plan(n, batch) as plan:
            assert S.sdft_schedule_describe(n, 0, idx).split(";")[0] in plan.describe()
            yr, yi = gpu_run(xr, xi, 0, plan=plan)
            assert rel_l2_rows(yr, yi, *O.dft_factored_dit(xr, xi)).max() <= TOL_F32
            zr, zi = gpu_run(xr, xi, 1, plan=plan, inplace=True)
            assert rel_l2_rows(zr, zi, *O.adjoint_factored(xr, xi)).max() <= TOL_F32
            assert plan.sync_status() == S.SDFT_OK
    finally:
        S.sdft_schedule_select(n, 0, prev)
