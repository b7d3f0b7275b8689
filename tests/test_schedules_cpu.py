"""Schedule candidates and the autotuner's bookkeeping (no GPU)."""
import json

import pytest

from paper_2504_07264_gb300 import autotune as A
from paper_2504_07264_gb300 import build as B
from paper_2504_07264_gb300 import sdft as S


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()


def test_every_length_has_schedules():
    for m in range(1, 17):
        n = 1 << m
        c = S.sdft_schedule_count(n, S.SDFT_F32)
        assert c >= 1
        names = [S.sdft_schedule_describe(n, S.SDFT_F32, i) for i in range(c)]
        assert all(f"N={n}:" in x for x in names)
        assert len(set(names)) == c
    assert S.sdft_schedule_count(256, S.SDFT_F32_SPLIT_BF16) == 1
    assert S.sdft_schedule_count(512, S.SDFT_F32_SPLIT_BF16) < 0
    assert S.sdft_schedule_count(1000, S.SDFT_F32) == -S.SDFT_ERR_UNSUPPORTED_N


def test_select_validates_and_sticks():
    n = 1024
    c = S.sdft_schedule_count(n, S.SDFT_F32)
    try:
        assert S.sdft_schedule_select(n, S.SDFT_F32, c) == S.SDFT_ERR_INVALID_ARG
        assert S.sdft_schedule_select(n, S.SDFT_F32, -1) == S.SDFT_ERR_INVALID_ARG
        assert S.sdft_schedule_select(n, S.SDFT_F32, c - 1) == S.SDFT_OK
        assert S.sdft_schedule_selected(n, S.SDFT_F32) == c - 1
    finally:
        S.sdft_schedule_select(n, S.SDFT_F32, 0)
    assert S.sdft_schedule_selected(n, S.SDFT_F32) == 0


def test_table_save_load_apply(tmp_path):
    path = str(tmp_path / "tune.json")
    rec = {"index": 1, "ms": [0.2, 0.1], "schedules": ["a", "b"]}
    A.save({"0": {"4096": rec}}, path, name="Test GPU")
    A.save({"0": {"2048": dict(rec, index=2)}}, path, name="Test GPU")
    table = A.load(path)
    assert set(table["Test GPU"]["0"]) == {"4096", "2048"}
    try:
        assert A.apply(table, name="Other GPU") == 0
        assert A.apply(table, name="Test GPU") == 2
        assert S.sdft_schedule_selected(4096, 0) == 1
        assert S.sdft_schedule_selected(2048, 0) == 2
    finally:
        S.sdft_schedule_select(4096, 0, 0)
        S.sdft_schedule_select(2048, 0, 0)


def test_shipped_table_is_valid_if_present():
    import os
    if not os.path.exists(A.SHIPPED):
        pytest.skip("no shipped tuning table")
    table = A.load(A.SHIPPED)
    for gpu, per_dtype in table.items():
        for dtype, per_n in per_dtype.items():
            for n, rec in per_n.items():
                if dtype == "ragged":
                    assert 0 <= rec < S.sdft_ragged_form_count(int(n)), (gpu, n)
                    continue
                assert 0 <= rec["index"] < S.sdft_schedule_count(int(n), int(dtype)), (gpu, n)
                json.dumps(rec)


def test_ragged_forms_save_apply(tmp_path):
    """The work-queue forms are kept beside the schedules and applied as the
    process-wide choice for later ragged plans."""
    path = str(tmp_path / "tune.json")
    A.save({"ragged": {"512": 1, "1024": 1}}, path, name="Test GPU")
    A.save({"0": {"4096": {"index": 0, "ms": [0.1], "schedules": ["a"]}}}, path, name="Test GPU")
    table = A.load(path)
    assert table["Test GPU"]["ragged"] == {"512": 1, "1024": 1}
    try:
        assert A.apply(table, name="Test GPU") == 3
        assert S.sdft_ragged_form_selected(512) == 1
        assert S.sdft_ragged_form_selected(1024) == 1
    finally:
        S.lib().sdft_ragged_form_select(512, 0)
        S.lib().sdft_ragged_form_select(1024, 0)
    # an out-of-range form in a table is skipped, not applied
    assert A.apply({"G": {"ragged": {"65536": 7}}}, name="G") == 0
