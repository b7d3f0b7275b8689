"""Ragged batches (GPU): mixed power-of-two lengths in one persistent launch
replayed from a CUDA graph, checked against the CPU oracle per transform."""
import numpy as np
import pytest

import workloads as W
from gpu_util import TOL_F32, rel_l2_rows
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available()
    from paper_2504_07264_gb300 import build
    build.build()
    O.build()


def _ragged_inputs(lengths, seed):
    rng = np.random.default_rng(seed)
    total = int(np.sum(lengths))
    xr = rng.standard_normal(total).astype(np.float32)
    xi = rng.standard_normal(total).astype(np.float32)
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(lengths, out=off[1:])
    return xr, xi, off


def _run(plan, xr, xi, direction, out=None):
    import torch
    dxr = torch.from_numpy(xr).cuda()
    dxi = torch.from_numpy(xi).cuda()
    if out is None:
        yr, yi = plan.execute(direction, dxr, dxi)
    else:
        yr, yi = plan.execute(direction, dxr, dxi, *out)
    torch.cuda.synchronize()
    return yr.cpu().numpy(), yi.cpu().numpy()


def _check_segments(lengths, off, xr, xi, yr, yi, direction, which=None):
    fn = O.dft_factored_dit if direction == 0 else O.adjoint_factored
    idx = range(len(lengths)) if which is None else which
    worst = 0.0
    for t in idx:
        a, b = off[t], off[t + 1]
        rr, ri = fn(xr[a:b][None, :], xi[a:b][None, :])
        e = rel_l2_rows(yr[a:b][None, :], yi[a:b][None, :], rr, ri).max()
        worst = max(worst, e)
    return worst


@pytest.mark.parametrize("direction", [0, 1])
def test_mixed_lengths_match_oracle(direction):
    from paper_2504_07264_gb300 import Plan
    rng = np.random.default_rng(40)
    lengths = (1 << rng.integers(2, 17, size=70)).astype(np.int64)
    lengths[:3] = [65536, 4, 32768]          # both two-pass classes and the smallest
    xr, xi, off = _ragged_inputs(lengths, 41 + direction)
    with Plan(lengths=lengths) as plan:
        assert plan.launches() == 1
        yr, yi = _run(plan, xr, xi, direction)
    assert _check_segments(lengths, off, xr, xi, yr, yi, direction) <= TOL_F32


def test_every_class_and_many_items():
    """Every length 4..65536, several work items per class, ragged counts."""
    from paper_2504_07264_gb300 import Plan
    lengths = []
    for logn in range(2, 17):
        reps = max(1, 3000 >> logn) + logn % 3
        lengths += [1 << logn] * reps
    lengths = np.random.default_rng(5).permutation(np.array(lengths, dtype=np.int64))
    xr, xi, off = _ragged_inputs(lengths, 43)
    with Plan(lengths=lengths) as plan:
        yr, yi = _run(plan, xr, xi, 0)
    pick = np.random.default_rng(6).choice(len(lengths), 80, replace=False)
    big = [t for t in range(len(lengths)) if lengths[t] >= 16384]
    assert _check_segments(lengths, off, xr, xi, yr, yi, 0, sorted(set(pick) | set(big))) <= TOL_F32


# uniform-plan schedule with the same arithmetic as the ragged kernel's form 0
# (the same radix split and tables; for N >= 16384 a cluster kernel with the
# same A x C split, whatever its number of CTAs)
SAME_SCHEDULE = {16: 0, 1024: 0, 4096: 0, 16384: 3, 32768: 3, 65536: 3}


def test_matches_uniform_plans_bitwise():
    """A ragged plan computes each transform exactly as the uniform plan of its
    length does on the schedule with the same radix split (same arithmetic and
    tables)."""
    from paper_2504_07264_gb300 import Plan
    from paper_2504_07264_gb300 import sdft as S
    for n, cnt in ((16, 700), (1024, 37), (4096, 9), (16384, 7), (32768, 5), (65536, 3)):
        lengths = np.full(cnt, n, dtype=np.int64)
        xr, xi, _ = _ragged_inputs(lengths, 44)
        with Plan(lengths=lengths) as rp:
            rp.set_ragged_form(n, 0)            # whatever the tuning table selected
            a = _run(rp, xr, xi, 0)
        prev = S.sdft_schedule_selected(n, 0)
        try:
            assert S.sdft_schedule_select(n, 0, SAME_SCHEDULE[n]) == S.SDFT_OK
            with Plan(n, cnt) as up:
                b = _run(up, xr.reshape(cnt, n), xi.reshape(cnt, n), 0)
        finally:
            S.sdft_schedule_select(n, 0, prev)
        assert np.array_equal(a[0], b[0].ravel()) and np.array_equal(a[1], b[1].ravel()), n


def test_bounded_wait_times_out_and_recovers():
    """A wait for a word that nothing sets (planted on the host) gives up: the
    status word reports SDFT_ERR_TIMEOUT, the kernel returns, and the same
    plan computes correctly afterwards."""
    import torch

    from paper_2504_07264_gb300 import Plan
    from paper_2504_07264_gb300 import sdft as S
    lengths = np.array([65536, 1024, 32768, 16384, 8], dtype=np.int64)
    xr, xi, off = _ragged_inputs(lengths, 47)
    with Plan(lengths=lengths) as plan:
        h = plan.handle
        assert S.sdft_plan_set_wait_limit(h, 2000) == S.SDFT_OK
        assert S.sdft_plan_inject_unreachable_wait(h, 1) == S.SDFT_OK
        _run(plan, xr, xi, 0)
        assert plan.sync_status() == S.SDFT_ERR_TIMEOUT
        assert S.sdft_plan_inject_unreachable_wait(h, 0) == S.SDFT_OK
        assert S.sdft_plan_set_wait_limit(h, 1 << 23) == S.SDFT_OK
        yr, yi = _run(plan, xr, xi, 0)
        assert plan.sync_status() == S.SDFT_OK
        torch.cuda.synchronize()
    assert _check_segments(lengths, off, xr, xi, yr, yi, 0) <= TOL_F32


def test_wait_hooks_reject_plans_without_waits():
    from paper_2504_07264_gb300 import Plan
    from paper_2504_07264_gb300 import sdft as S
    with Plan(1024, 4) as plan:
        assert S.sdft_plan_set_wait_limit(plan.handle, 10) == S.SDFT_ERR_INVALID_ARG
        assert S.sdft_plan_inject_unreachable_wait(plan.handle, 1) == S.SDFT_ERR_INVALID_ARG
    with Plan(lengths=np.array([8, 1024], dtype=np.int64)) as plan:
        assert S.sdft_plan_inject_unreachable_wait(plan.handle, 1) == S.SDFT_ERR_INVALID_ARG


def test_graph_replay_with_new_buffers():
    import torch

    from paper_2504_07264_gb300 import Plan
    lengths = np.array([8, 1024, 65536, 64, 4096, 16], dtype=np.int64)
    xr, xi, off = _ragged_inputs(lengths, 45)
    with Plan(lengths=lengths) as plan:
        first = _run(plan, xr, xi, 0)
        out = (torch.empty(xr.size, device="cuda"), torch.empty(xr.size, device="cuda"))
        second = _run(plan, xr, xi, 0, out=out)     # new input and output pointers
        third = _run(plan, xr, xi, 0)               # and back
    for r in (second, third):
        assert np.array_equal(first[0], r[0]) and np.array_equal(first[1], r[1])
    assert _check_segments(lengths, off, xr, xi, *first, 0) <= TOL_F32


def test_in_place_and_host_buffers():
    import torch

    from paper_2504_07264_gb300 import Plan
    lengths = np.array([65536, 8, 2048, 32768, 4], dtype=np.int64)
    xr, xi, off = _ragged_inputs(lengths, 46)
    with Plan(lengths=lengths) as plan:
        ref = _run(plan, xr, xi, 1)
        dxr = torch.from_numpy(xr).cuda()
        dxi = torch.from_numpy(xi).cuda()
        plan.execute(1, dxr, dxi, dxr, dxi)
        torch.cuda.synchronize()
        assert np.array_equal(dxr.cpu().numpy(), ref[0]) and np.array_equal(dxi.cpu().numpy(), ref[1])
        hyr = np.empty_like(xr)
        hyi = np.empty_like(xi)
        plan.execute_host(1, xr, xi, hyr, hyi)
        assert np.array_equal(hyr, ref[0]) and np.array_equal(hyi, ref[1])


def test_full_ragged_workload_sampled():
    """10000 transforms, lengths 2^U{3..16} (seed 4): sampled transforms of every
    length against the oracle, Parseval on every transform."""
    import torch

    from paper_2504_07264_gb300 import Plan
    lengths, off, xr, xi = W.ragged_planes()
    assert int(off[-1]) == 96714152
    with Plan(lengths=lengths) as plan:
        dxr = torch.from_numpy(xr).cuda()
        dxi = torch.from_numpy(xi).cuda()
        yr, yi = plan.forward(dxr, dxi)
        seg = torch.repeat_interleave(torch.arange(len(lengths), device="cuda"),
                                      torch.from_numpy(lengths).cuda())
        e_in = torch.zeros(len(lengths), dtype=torch.float64, device="cuda").index_add_(
            0, seg, dxr.double() ** 2 + dxi.double() ** 2) * torch.from_numpy(lengths).cuda()
        e_out = torch.zeros(len(lengths), dtype=torch.float64, device="cuda").index_add_(
            0, seg, yr.double() ** 2 + yi.double() ** 2)
        parseval = ((e_out - e_in).abs() / e_in).max().item()
        hy = (yr.cpu().numpy(), yi.cpu().numpy())
    assert parseval < 1e-5
    rng = np.random.default_rng(7)
    pick = []
    for logn in range(3, 17):
        cand = np.nonzero(lengths == (1 << logn))[0]
        pick += list(rng.choice(cand, min(2, cand.size), replace=False))
    assert _check_segments(lengths, off, xr, xi, *hy, 0, sorted(pick)) <= TOL_F32


def test_every_form_matches_oracle():
    """Every compiled form of every length (row tiles of each radix split and
    tile size, transforms held by 8, 4 or 2 CTAs) against the oracle, in both
    directions, in one plan holding every length; the form switch rebuilds
    the plan's work items between calls."""
    from paper_2504_07264_gb300 import Plan
    from paper_2504_07264_gb300 import sdft as S
    lengths = np.array([1 << l for l in range(2, 17) for _ in range(3 + (l < 12) * 9)],
                       dtype=np.int64)
    lengths = np.random.default_rng(48).permutation(lengths)
    xr, xi, off = _ragged_inputs(lengths, 48)
    with Plan(lengths=lengths) as plan:
        for logn in range(2, 17):
            n = 1 << logn
            # a new plan starts with the process-wide selection (the tuning table's)
            assert plan.ragged_form(n) == S.sdft_ragged_form_selected(n)
            which = [t for t in range(len(lengths)) if lengths[t] == n]
            for f in range(S.sdft_ragged_form_count(n)):
                plan.set_ragged_form(n, f)
                assert plan.ragged_form(n) == f
                for direction in (0, 1):
                    yr, yi = _run(plan, xr, xi, direction)
                    err = _check_segments(lengths, off, xr, xi, yr, yi, direction, which)
                    assert err <= TOL_F32, (n, f, direction, err)
                assert plan.sync_status() == S.SDFT_OK
            plan.set_ragged_form(n, 0)
        with pytest.raises(S.SdftError):
            plan.set_ragged_form(1024, S.sdft_ragged_form_count(1024))
    with Plan(lengths=np.array([8, 1024], dtype=np.int64)) as plan:
        with pytest.raises(S.SdftError):
            plan.set_ragged_form(4096, 0)          # a length the plan does not hold
    with Plan(1024, 4) as uplan:
        with pytest.raises(S.SdftError):
            uplan.set_ragged_form(1024, 0)


def test_groups_of_every_size_in_one_launch():
    """Forms that put transforms on groups of 8, 4 and 2 CTAs and on row tiles
    in the same plan, with more transforms than groups in every phase, so that
    groups split and finish at different times, and the last round of each
    group phase leaves some groups of a cluster without a transform."""
    from paper_2504_07264_gb300 import Plan
    from paper_2504_07264_gb300 import sdft as S
    rng = np.random.default_rng(49)
    lengths = np.concatenate([np.full(c, n, np.int64) for n, c in
                              ((65536, 45), (32768, 70), (16384, 150), (8192, 200), (512, 900))])
    lengths = rng.permutation(lengths)
    xr, xi, off = _ragged_inputs(lengths, 49)
    # N = 65536 and 32768 on eight CTAs, 16384 on four, 8192 on two; 512 in
    # each of its row forms
    for f9 in range(S.sdft_ragged_form_count(512)):
        with Plan(lengths=lengths) as plan:
            plan.set_ragged_form(512, f9)
            for direction in (0, 1):
                yr, yi = _run(plan, xr, xi, direction)
                assert plan.sync_status() == S.SDFT_OK
                pick = sorted(set(rng.choice(len(lengths), 60, replace=False)) |
                              {int(np.argmax(lengths == n)) for n in (65536, 32768, 16384, 8192)})
                assert _check_segments(lengths, off, xr, xi, yr, yi, direction, pick) <= TOL_F32


def test_ragged_autotune_keeps_valid_forms():
    import torch

    from paper_2504_07264_gb300 import Plan
    from paper_2504_07264_gb300 import sdft as S
    lengths = np.array([1 << l for l in range(2, 17) for _ in range(4)], dtype=np.int64)
    lengths = np.random.default_rng(50).permutation(lengths)
    xr, xi, off = _ragged_inputs(lengths, 50)
    with Plan(lengths=lengths) as plan:
        dxr, dxi = torch.from_numpy(xr).cuda(), torch.from_numpy(xi).cuda()
        m = plan.ragged_autotune(dxr, dxi, torch.empty_like(dxr), torch.empty_like(dxi), reps=2)
        assert m >= 0
        for logn in range(2, 17):
            f = plan.ragged_form(1 << logn)
            assert 0 <= f < S.sdft_ragged_form_count(1 << logn)
            assert bool(m >> logn & 1) == (f != 0)
        yr, yi = _run(plan, xr, xi, 0)
        assert _check_segments(lengths, off, xr, xi, yr, yi, 0) <= TOL_F32


@pytest.mark.parametrize("lengths", [[65536], [32768], [16384], [8192], [4096], [4],
                                     [65536, 4], [4, 8, 16]])
def test_one_transform_per_class(lengths):
    """Plans of one or two transforms: every phase but one has no items, and
    all groups or CTAs but one of the persistent grid find nothing to do (they
    take the cluster barriers only, or claim no row tile) and the call still
    ends, with each transform right in both directions."""
    from paper_2504_07264_gb300 import Plan
    lengths = np.array(lengths, dtype=np.int64)
    xr, xi, off = _ragged_inputs(lengths, 70 + int(lengths.sum() % 97))
    with Plan(lengths=lengths) as plan:
        for direction in (0, 1):
            yr, yi = _run(plan, xr, xi, direction)
            assert _check_segments(lengths, off, xr, xi, yr, yi, direction) <= TOL_F32
        assert plan.sync_status() == 0
