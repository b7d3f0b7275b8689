"""The C ABI library builds, loads and exports every declared symbol; host-side
argument checks work without a GPU (no compute call is made here)."""
import ctypes
import re
import subprocess

import pytest

from paper_2504_07264_gb300 import build as B
from paper_2504_07264_gb300 import sdft as S


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def test_exports_every_header_symbol():
    names = S.header_symbols()
    assert len(names) >= 15
    lib = ctypes.CDLL(S.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"
    # and nothing else leaks out of the library as a dynamic symbol
    out = subprocess.run(["nm", "-D", "--defined-only", S.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert set(names) <= exported
    assert all(not n.startswith("_ZN4sdft") for n in exported)


def test_binding_covers_header():
    assert set(S.header_symbols()) == set(S._SIGS)


def test_header_constants_match_binding():
    with open(S.HEADER) as f:
        text = f.read()
    defs = dict(re.findall(r"#define\s+(SDFT_\w+)\s+(-?\d+)", text))
    assert defs, "no constants parsed"
    for name, val in defs.items():
        assert getattr(S, name) == int(val), name


def test_version_and_status_strings():
    assert re.fullmatch(r"\d+\.\d+\.\d+", S.sdft_version())
    for code in range(10):
        assert S.sdft_status_string(code)
    assert S.sdft_status_string(0) == "ok"
    assert "unknown" in S.sdft_status_string(999)


@pytest.mark.parametrize("n", [0, 1, 3, 6, 1000, 1 << 17, -4])
def test_unsupported_length_rejected_before_cuda(n):
    assert S.sdft_plan_create(n, 4, S.SDFT_F32) == 0
    assert S.sdft_last_error() == S.SDFT_ERR_UNSUPPORTED_N


@pytest.mark.parametrize("batch", [0, -1])
def test_bad_batch_rejected(batch):
    assert S.sdft_plan_create(1024, batch, S.SDFT_F32) == 0
    assert S.sdft_last_error() == S.SDFT_ERR_INVALID_ARG


def test_bad_dtype_rejected():
    assert S.sdft_plan_create(1024, 4, 7) == 0
    assert S.sdft_last_error() == S.SDFT_ERR_UNSUPPORTED_DTYPE
    # the split tensor-core path exists for N = 256 and 1024 only
    for n in (16, 512, 2048):
        for dt in (S.SDFT_F32_SPLIT_BF16, S.SDFT_F32_SPLIT_FP16):
            assert S.sdft_plan_create(n, 4, dt) == 0
            assert S.sdft_last_error() == S.SDFT_ERR_UNSUPPORTED_DTYPE


@pytest.mark.parametrize("handle", [0, 12345678, 0xDEADBEEF0])
def test_bad_plan_handles(handle):
    assert S.sdft_forward(handle, 16, 16, 16, 16, 0) == S.SDFT_ERR_BAD_PLAN
    assert S.sdft_adjoint(handle, 16, 16, 16, 16, 0) == S.SDFT_ERR_BAD_PLAN
    assert S.sdft_execute(handle, 0, 16, 16, 16, 16, 0) == S.SDFT_ERR_BAD_PLAN
    assert S.sdft_execute_host(handle, 0, 16, 16, 16, 16, 0) == S.SDFT_ERR_BAD_PLAN
    assert S.sdft_plan_sync_status(handle, 0) == S.SDFT_ERR_BAD_PLAN
    assert S.sdft_plan_set_ragged_form(handle, 1024, 0) == S.SDFT_ERR_BAD_PLAN
    assert S.sdft_plan_ragged_form(handle, 1024) == -S.SDFT_ERR_BAD_PLAN
    assert S.sdft_plan_ragged_autotune(handle, 16, 16, 16, 16, 1, 0) == -S.SDFT_ERR_BAD_PLAN
    assert S.sdft_last_error() == S.SDFT_ERR_BAD_PLAN
    assert S.sdft_plan_n(handle) == 0 and S.sdft_plan_launches(handle, 0) == 0
    S.sdft_plan_destroy(handle)  # foreign handles are ignored, not freed


def test_ragged_rejects_bad_lengths_before_cuda():
    import numpy as np
    for lengths in ([8, 12], [8, 2], [], [1 << 17]):
        arr = np.asarray(lengths, dtype=np.int64)
        h = S.sdft_plan_create_ragged(arr.ctypes.data if arr.size else 0, arr.size, S.SDFT_F32)
        assert h == 0
        assert S.sdft_last_error() in (S.SDFT_ERR_UNSUPPORTED_N, S.SDFT_ERR_INVALID_ARG)


def test_ragged_forms_catalogue():
    """Every length 4 .. 65536 has at least one work-queue form; form 0 is the
    default; out-of-range lengths and forms are rejected on the host."""
    for logn in range(2, 17):
        n = 1 << logn
        c = S.sdft_ragged_form_count(n)
        assert c >= 1
        for f in range(c):
            assert S.sdft_ragged_form_describe(n, f).startswith(f"N={n}:")
        assert S.lib().sdft_ragged_form_describe(n, c, None, 0) == -S.SDFT_ERR_INVALID_ARG
    # lengths with a choice of radix split and tile size for the plan tuner
    for n in (256, 512, 1024, 2048):
        assert S.sdft_ragged_form_count(n) >= 2
    for n in (2, 3, 131072):
        assert S.sdft_ragged_form_count(n) == -S.SDFT_ERR_UNSUPPORTED_N
    assert S.lib().sdft_ragged_form_select(1024, 99) == S.SDFT_ERR_INVALID_ARG
    assert S.lib().sdft_ragged_form_select(2, 0) == S.SDFT_ERR_UNSUPPORTED_N


def _layout_invariants(lengths):
    import numpy as np
    phase, item, nitems = S.sdft_ragged_work_layout(lengths)
    n = len(lengths)
    assert phase.shape == (n,) and ((phase >= 0) & (phase <= 3)).all()
    for ph in range(4):
        sel = np.nonzero(phase == ph)[0]
        if ph < 3:
            # one transform per group item, every item used once, and the CTAs
            # per transform of the form match the phase (8, 4, 2)
            assert sorted(item[sel]) == list(range(nitems[ph]))
            q = {0: 8, 1: 4, 2: 2}[ph]
            for t in sel:
                f = S.sdft_ragged_form_selected(int(lengths[t]))
                assert f"{q} CTAs" in S.sdft_ragged_form_describe(int(lengths[t]), f)
        else:
            assert set(item[sel]) == set(range(nitems[3]))
            for it in range(nitems[3]):
                members = lengths[sel[item[sel] == it]]
                assert members.size >= 1 and (members == members[0]).all()
        # items of a phase are ordered longest transforms first
        if sel.size:
            first_len = [lengths[sel[item[sel] == it][0]] for it in range(nitems[ph])]
            assert all(a >= b for a, b in zip(first_len, first_len[1:]))
    return phase, item, nitems


def test_ragged_work_layout_host_logic():
    """The ragged plan's work items, computed on the host (no GPU): every
    transform in exactly one item of the phase its length's form puts it in,
    group items one transform each, row tiles of one length, longest first."""
    import numpy as np
    rng = np.random.default_rng(60)
    for trial in range(5):
        lengths = (1 << rng.integers(2, 17, size=300 + 100 * trial)).astype(np.int64)
        _layout_invariants(lengths)
    # the benchmark's workload: lengths 2^U{3..16}, seed 4
    import workloads
    cfg = workloads.RAGGED
    lengths, _ = workloads.ragged_lengths(cfg["count"], cfg["kmin"], cfg["kmax"], cfg["seed"])
    phase, item, nitems = _layout_invariants(lengths)
    assert nitems.sum() == (phase < 3).sum() + nitems[3]


def test_ragged_work_layout_follows_forms_and_rejects_bad_lengths():
    import numpy as np
    lengths = np.array([512] * 20 + [8192, 4], dtype=np.int64)
    try:
        for f in range(S.sdft_ragged_form_count(512)):
            assert S.lib().sdft_ragged_form_select(512, f) == S.SDFT_OK
            per = int(S.sdft_ragged_form_describe(512, f).split("tile of ")[1].split()[0])
            phase, item, nitems = _layout_invariants(lengths)
            rows512 = item[(lengths == 512)]
            assert len(set(rows512)) == -(-20 // per)
    finally:
        S.lib().sdft_ragged_form_select(512, 0)
    for bad in ([8, 12], [2], [1 << 17]):
        with pytest.raises(S.SdftError):
            S.sdft_ragged_work_layout(np.asarray(bad, dtype=np.int64))
