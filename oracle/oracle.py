"""CPU oracle for the split (planar) complex DFT -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this module.  The CUDA library never imports it, and
it imports nothing from the CUDA library.

This module compiles ``sdft_oracle.c`` (plain C, binary64, no fast-math, no FMA
contraction) with gcc and exposes its entry points on numpy float64 arrays.
See the C file's header for which equation of the paper each function follows:

  dft_direct          Eq. (1) in the split form of Eq. (3)          (O1)
  dft_direct_bins     the same, on chosen bins                      (O1b)
  dft_factored_dit    the vector-matrix procedure Eq. (6)           (O2)
  dit_stages          Eq. (6) on one transform, every intermediate  (O2s)
  adjoint_direct      transpose of the block matrix Eq. (5)         (O3)
  adjoint_factored    transpose of the Eq. (6) product              (O3f)
  dft_factored_dif    the decimation-in-frequency procedure Eq. (9) (O4)
  dft_factored_dit_f32  Eq. (6) in binary32 (CPU baseline's FP32 instance) (O2f)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdft_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict[int, ctypes.CDLL] = {}

_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I64P = ctypes.POINTER(ctypes.c_int64)


def lib_path(mutation: int = 0) -> str:
    name = "liboracle.so" if mutation == 0 else f"liboracle_mut{mutation}.so"
    return os.path.join(_BUILD, name)


def build(mutation: int = 0, force: bool = False) -> str:
    """Compile the oracle (or a copy with planted mistake ``mutation``)."""
    out = lib_path(mutation)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)):
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math",
           f"-DSDFT_ORACLE_MUTATION={int(mutation)}", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _load(mutation: int = 0) -> ctypes.CDLL:
    with _LOCK:
        lib = _LIBS.get(mutation)
        if lib is not None:
            return lib
        lib = ctypes.CDLL(build(mutation))
        sig5 = [ctypes.c_int64, ctypes.c_int64, _D, _D, _D, _D, ctypes.c_int]
        for name in ("sdft_oracle_direct", "sdft_oracle_factored_dit",
                     "sdft_oracle_factored_dif", "sdft_oracle_adjoint_direct",
                     "sdft_oracle_adjoint_factored"):
            f = getattr(lib, name)
            f.argtypes = sig5
            f.restype = ctypes.c_int
        lib.sdft_oracle_direct_bins.argtypes = [
            ctypes.c_int64, ctypes.c_int64, _D, _D, _I64P, ctypes.c_int64, _D, _D,
            ctypes.c_int]
        lib.sdft_oracle_direct_bins.restype = ctypes.c_int
        lib.sdft_oracle_dit_stages.argtypes = [ctypes.c_int64, _D, _D]
        lib.sdft_oracle_dit_stages.restype = ctypes.c_int
        lib.sdft_oracle_factored_dit_f32.argtypes = [ctypes.c_int64, ctypes.c_int64, _F, _F, _F,
                                                     _F, ctypes.c_int]
        lib.sdft_oracle_factored_dit_f32.restype = ctypes.c_int
        lib.sdft_oracle_thread_count.argtypes = [ctypes.c_int]
        lib.sdft_oracle_thread_count.restype = ctypes.c_int
        _LIBS[mutation] = lib
        return lib


def _as_rows(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(1, -1) if a.ndim == 1 else a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _batched(name: str, xr, xi, threads: int, mutation: int):
    squeeze = np.ndim(xr) == 1
    xr = _as_rows(xr)
    xi = _as_rows(xi)
    if xr.shape != xi.shape:
        raise ValueError("xr and xi must have the same shape")
    batch, n = xr.shape
    yr = np.empty_like(xr)
    yi = np.empty_like(xi)
    rc = getattr(_load(mutation), name)(n, batch, _ptr(xr), _ptr(xi), _ptr(yr), _ptr(yi),
                                        int(threads))
    if rc != 0:
        raise ValueError(f"{name}: rejected n={n} batch={batch} (rc={rc})")
    if squeeze:
        return yr[0], yi[0]
    return yr, yi


def dft_direct(xr, xi, threads: int = 0, mutation: int = 0):
    """O1: Eq. (1)/(3), direct O(N^2) sum in binary64."""
    return _batched("sdft_oracle_direct", xr, xi, threads, mutation)


def dft_factored_dit(xr, xi, threads: int = 0, mutation: int = 0):
    """O2: the procedure of Eq. (6), N = 2^m."""
    return _batched("sdft_oracle_factored_dit", xr, xi, threads, mutation)


def dft_factored_dit_f32(xr, xi, threads: int = 0):
    """O2f: the procedure of Eq. (6) in binary32 on float32 rows (the CPU
    baseline's single-precision instance; checked against O2)."""
    squeeze = np.ndim(xr) == 1
    xr = np.ascontiguousarray(xr, dtype=np.float32)
    xi = np.ascontiguousarray(xi, dtype=np.float32)
    xr = xr.reshape(1, -1) if xr.ndim == 1 else xr
    xi = xi.reshape(1, -1) if xi.ndim == 1 else xi
    if xr.shape != xi.shape:
        raise ValueError("xr and xi must have the same shape")
    batch, n = xr.shape
    yr = np.empty_like(xr)
    yi = np.empty_like(xi)
    f = _load(0).sdft_oracle_factored_dit_f32
    rc = f(n, batch, xr.ctypes.data_as(_F), xi.ctypes.data_as(_F), yr.ctypes.data_as(_F),
           yi.ctypes.data_as(_F), int(threads))
    if rc != 0:
        raise ValueError(f"sdft_oracle_factored_dit_f32: rejected n={n} batch={batch} (rc={rc})")
    if squeeze:
        return yr[0], yi[0]
    return yr, yi


def dft_factored_dif(xr, xi, threads: int = 0, mutation: int = 0):
    """O4: the procedure of Eq. (9), N = 2^m."""
    return _batched("sdft_oracle_factored_dif", xr, xi, threads, mutation)


def adjoint_direct(xr, xi, threads: int = 0, mutation: int = 0):
    """O3: E_2N^T of Eq. (5) applied directly (the conjugate-transpose DFT)."""
    return _batched("sdft_oracle_adjoint_direct", xr, xi, threads, mutation)


def adjoint_factored(xr, xi, threads: int = 0, mutation: int = 0):
    """O3f: transpose of the Eq. (6) product, factor by factor."""
    return _batched("sdft_oracle_adjoint_factored", xr, xi, threads, mutation)


def dft_direct_bins(xr, xi, bins, threads: int = 0, mutation: int = 0):
    """O1b: Eq. (3) on the bins ``bins`` of every transform -> (batch, nbins)."""
    xr = _as_rows(xr)
    xi = _as_rows(xi)
    bins = np.ascontiguousarray(bins, dtype=np.int64)
    batch, n = xr.shape
    yr = np.empty((batch, bins.size))
    yi = np.empty((batch, bins.size))
    rc = _load(mutation).sdft_oracle_direct_bins(
        n, batch, _ptr(xr), _ptr(xi), bins.ctypes.data_as(_I64P), bins.size,
        _ptr(yr), _ptr(yi), int(threads))
    if rc != 0:
        raise ValueError(f"dft_direct_bins: rejected n={n} (rc={rc})")
    return yr, yi


def dit_stages(x2, mutation: int = 0) -> np.ndarray:
    """O2s: Eq. (6) on one interleaved pair vector x_2N (Section III).

    Returns an array of shape (2m+1, 2N): row 0 is S x, rows 2i-1 and 2i are
    the vector after D(i) and after W(i).
    """
    x2 = np.ascontiguousarray(x2, dtype=np.float64)
    n = x2.size // 2
    m = n.bit_length() - 1
    out = np.empty((2 * m + 1, 2 * n))
    rc = _load(mutation).sdft_oracle_dit_stages(n, _ptr(x2), _ptr(out))
    if rc != 0:
        raise ValueError(f"dit_stages: rejected n={n}")
    return out


def thread_count(threads: int = 0) -> int:
    """OpenMP threads a call with ``threads`` uses."""
    return int(_load().sdft_oracle_thread_count(int(threads)))


def default_threads() -> int:
    return os.cpu_count() or 1
