"""Seeded synthetic inputs for the split complex DFT.

This module is shared by the tests, the benchmark and the smoke check.  It
holds only random-number draws and shapes -- none of the transform's
arithmetic -- so the CUDA path and the CPU oracle share no computation through
it.  Every generator uses ``numpy.random.default_rng(seed)``, draws in binary64
in the order documented per function, and returns C-contiguous float32 planes
(the values the GPU sees; the oracle upcasts these same float32 values).

Workloads (the paper has no datasets or experiments; these are synthetic
stand-ins with the shapes and value distributions of the measured configs):

  plain      1024 transforms of N = 16, entries iid U[-1, 1), seed 0
  bandwidth  65536 transforms of N = 1024, iid N(0, 1), seed 1
  autograd   16384 transforms of N = 4096, iid N(0, 1), seed 1, plus loss
             weights w_r, w_i iid U[0, 1) of the same shape, seed 2
  precision  262144 transforms of N = 256, |x| = 10^U(-3, 3), phase U[0, 2pi),
             seed 3 (magnitudes drawn first, then phases)
  ragged     10000 transforms of lengths 2^k, k uniform in {3..16}, seed 4
             (lengths drawn first, then data iid N(0, 1))
  integer    integer-valued entries uniform in [-8, 8], seed 5
"""
from __future__ import annotations

import numpy as np

PLAIN = dict(n=16, batch=1024, seed=0)
BANDWIDTH = dict(n=1024, batch=65536, seed=1)
AUTOGRAD = dict(n=4096, batch=16384, seed=1, weight_seed=2)
PRECISION = dict(n=256, batch=262144, seed=3)
RAGGED = dict(count=10000, kmin=3, kmax=16, seed=4)
INTEGER_SEED = 5


def _f32(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def uniform_planes(n: int, batch: int, seed: int, lo: float = -1.0, hi: float = 1.0):
    """xr then xi, each (batch, n), iid U[lo, hi)."""
    rng = np.random.default_rng(seed)
    xr = rng.uniform(lo, hi, size=(batch, n))
    xi = rng.uniform(lo, hi, size=(batch, n))
    return _f32(xr), _f32(xi)


def normal_planes(n: int, batch: int, seed: int):
    """xr then xi, each (batch, n), iid standard normal."""
    rng = np.random.default_rng(seed)
    xr = rng.standard_normal(size=(batch, n))
    xi = rng.standard_normal(size=(batch, n))
    return _f32(xr), _f32(xi)


def integer_planes(n: int, batch: int, seed: int = INTEGER_SEED, bound: int = 8):
    """xr then xi, each (batch, n), integers uniform in [-bound, bound]."""
    rng = np.random.default_rng(seed)
    xr = rng.integers(-bound, bound + 1, size=(batch, n))
    xi = rng.integers(-bound, bound + 1, size=(batch, n))
    return _f32(xr), _f32(xi)


def logmag_phase_planes(n: int, batch: int, seed: int, lo_exp: float = -3.0,
                        hi_exp: float = 3.0):
    """|x| = 10^U(lo_exp, hi_exp) drawn first, then phase U[0, 2 pi)."""
    rng = np.random.default_rng(seed)
    mag = 10.0 ** rng.uniform(lo_exp, hi_exp, size=(batch, n))
    phase = rng.uniform(0.0, 2.0 * np.pi, size=(batch, n))
    return _f32(mag * np.cos(phase)), _f32(mag * np.sin(phase))


def loss_weights(n: int, batch: int, seed: int):
    """w_r then w_i, each (batch, n), iid U[0, 1)."""
    rng = np.random.default_rng(seed)
    wr = rng.uniform(0.0, 1.0, size=(batch, n))
    wi = rng.uniform(0.0, 1.0, size=(batch, n))
    return _f32(wr), _f32(wi)


def ragged_lengths(count: int, kmin: int, kmax: int, seed: int):
    """Lengths 2^k with k uniform in {kmin..kmax}; returns (lengths, rng)."""
    rng = np.random.default_rng(seed)
    k = rng.integers(kmin, kmax + 1, size=count)
    return (np.int64(1) << k.astype(np.int64)), rng


def ragged_planes(count: int = RAGGED["count"], kmin: int = RAGGED["kmin"],
                  kmax: int = RAGGED["kmax"], seed: int = RAGGED["seed"]):
    """Ragged batch: lengths first, then xr then xi (concatenated rows) iid N(0, 1).

    Returns (lengths int64[count], offsets int64[count+1], xr, xi) where
    transform t occupies [offsets[t], offsets[t+1]) of the flat planes.
    """
    lengths, rng = ragged_lengths(count, kmin, kmax, seed)
    offsets = np.zeros(count + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    total = int(offsets[-1])
    xr = rng.standard_normal(size=total)
    xi = rng.standard_normal(size=total)
    return lengths, offsets, _f32(xr), _f32(xi)


def plain():
    return uniform_planes(PLAIN["n"], PLAIN["batch"], PLAIN["seed"])


def bandwidth(batch: int | None = None):
    b = BANDWIDTH["batch"] if batch is None else batch
    return normal_planes(BANDWIDTH["n"], b, BANDWIDTH["seed"])


def precision(batch: int | None = None):
    b = PRECISION["batch"] if batch is None else batch
    return logmag_phase_planes(PRECISION["n"], b, PRECISION["seed"])
