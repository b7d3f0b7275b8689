"""The binary32 instance of the Eq. (6) procedure (the CPU baseline's FP32
leg), pinned to the binary64 oracle and to exact cases (CPU only)."""
import numpy as np
import pytest

import workloads as W
from oracle import oracle as O


@pytest.fixture(scope="module", autouse=True)
def _built():
    O.build()


@pytest.mark.parametrize("logn", [1, 2, 3, 5, 6, 8, 10, 12])
def test_f32_instance_tracks_the_float64_procedure(logn):
    n = 1 << logn
    xr, xi = W.normal_planes(n, 9, seed=70 + logn)
    yr, yi = O.dft_factored_dit_f32(xr, xi)
    assert yr.dtype == np.float32 and yr.shape == xr.shape
    rr, ri = O.dft_factored_dit(xr.astype(np.float64), xi.astype(np.float64))
    err = np.sqrt(((yr - rr) ** 2 + (yi - ri) ** 2).sum(1) / (rr ** 2 + ri ** 2).sum(1))
    # binary32 rounding over log2(N) stages: a few 1e-7, far below 1e-6
    assert err.max() < 5e-7, err.max()


@pytest.mark.parametrize("n", [2, 4, 16, 256])
def test_f32_instance_delta_gives_ones_exactly(n):
    xr = np.zeros((1, n), np.float32)
    xi = np.zeros((1, n), np.float32)
    xr[0, 0] = 1.0
    yr, yi = O.dft_factored_dit_f32(xr, xi)
    assert np.array_equal(yr, np.ones((1, n), np.float32))
    assert np.array_equal(yi, np.zeros((1, n), np.float32))


@pytest.mark.parametrize("n", [2, 4])
def test_f32_instance_exact_on_small_integers(n):
    rng = np.random.default_rng(5)
    xr = rng.integers(-8, 9, (6, n)).astype(np.float32)
    xi = rng.integers(-8, 9, (6, n)).astype(np.float32)
    yr, yi = O.dft_factored_dit_f32(xr, xi)
    rr, ri = O.dft_factored_dit(xr.astype(np.float64), xi.astype(np.float64))
    assert np.array_equal(yr.astype(np.float64), rr) and np.array_equal(yi.astype(np.float64), ri)


def test_f32_instance_rejects_non_power_of_two():
    x = np.zeros((2, 12), np.float32)
    with pytest.raises(ValueError):
        O.dft_factored_dit_f32(x, x)
