"""Python binding of the C ABI in ``include/sdft.h`` (libsdft.so).

The ``sdft_*`` functions below carry the C entry points' names and arguments
(raw integers for pointers, plans and streams) and do argument marshalling
only: every step of the transform runs in the CUDA kernels of libsdft.so.
``Plan`` wraps them for torch tensors: it checks dtype/device/layout, passes
the tensors' device pointers and torch's current CUDA stream, and raises
``SdftError`` on any non-OK status.

There is no fallback: if libsdft.so has not been built, importing the
library raises.  Build it with ``python -m paper_2504_07264_gb300.build``.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsdft.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "sdft.h")

# status codes and constants (mirroring include/sdft.h)
SDFT_OK = 0
SDFT_ERR_INVALID_ARG = 1
SDFT_ERR_UNSUPPORTED_N = 2
SDFT_ERR_MISALIGNED = 3
SDFT_ERR_ALIAS = 4
SDFT_ERR_BAD_PLAN = 5
SDFT_ERR_CUDA = 6
SDFT_ERR_ALLOC = 7
SDFT_ERR_TIMEOUT = 8
SDFT_ERR_UNSUPPORTED_DTYPE = 9
SDFT_F32 = 0
SDFT_F32_SPLIT_BF16 = 1
SDFT_F32_SPLIT_FP16 = 2
SDFT_FORWARD = 0
SDFT_ADJOINT = 1
SDFT_HOST_AUTO = 0
SDFT_HOST_STAGED = 1
SDFT_HOST_ZERO_COPY = 2

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGS = {
    "sdft_plan_create": ([_I64, _I64, ctypes.c_int], _P),
    "sdft_plan_create_ragged": ([_P, _I64, ctypes.c_int], _P),
    "sdft_plan_destroy": ([_P], None),
    "sdft_forward": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "sdft_adjoint": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "sdft_execute": ([_P, ctypes.c_int, _P, _P, _P, _P, _P], ctypes.c_int),
    "sdft_execute_host": ([_P, ctypes.c_int, _P, _P, _P, _P, _P], ctypes.c_int),
    "sdft_plan_sync_status": ([_P, _P], ctypes.c_int),
    "sdft_plan_set_host_mode": ([_P, ctypes.c_int], ctypes.c_int),
    "sdft_plan_set_grid": ([_P, ctypes.c_int], ctypes.c_int),
    "sdft_plan_set_wait_limit": ([_P, ctypes.c_int], ctypes.c_int),
    "sdft_ragged_form_count": ([_I64], ctypes.c_int),
    "sdft_ragged_form_describe": ([_I64, ctypes.c_int, ctypes.c_char_p, _I64], ctypes.c_int),
    "sdft_ragged_form_select": ([_I64, ctypes.c_int], ctypes.c_int),
    "sdft_ragged_form_selected": ([_I64], ctypes.c_int),
    "sdft_plan_set_ragged_form": ([_P, _I64, ctypes.c_int], ctypes.c_int),
    "sdft_plan_ragged_form": ([_P, _I64], ctypes.c_int),
    "sdft_ragged_work_layout": ([_P, _I64, _P, _P, _P], ctypes.c_int),
    "sdft_plan_ragged_autotune": ([_P, _P, _P, _P, _P, ctypes.c_int, _P], ctypes.c_int),
    "sdft_plan_inject_unreachable_wait": ([_P, ctypes.c_int], ctypes.c_int),
    "sdft_plan_grid": ([_P], ctypes.c_int),
    "sdft_execute_noalloc": ([_I64, _I64, ctypes.c_int, _P, _P, _P, _P, _P], ctypes.c_int),
    "sdft_schedule_count": ([_I64, ctypes.c_int], ctypes.c_int),
    "sdft_schedule_describe": ([_I64, ctypes.c_int, ctypes.c_int, ctypes.c_char_p, _I64], ctypes.c_int),
    "sdft_schedule_select": ([_I64, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "sdft_schedule_selected": ([_I64, ctypes.c_int], ctypes.c_int),
    "sdft_autotune": ([_I64, _I64, ctypes.c_int, _P, _P, _P, _P, ctypes.c_int, _P, _P], ctypes.c_int),
    "sdft_plan_n": ([_P], _I64),
    "sdft_plan_batch": ([_P], _I64),
    "sdft_plan_points": ([_P], _I64),
    "sdft_plan_dtype": ([_P], ctypes.c_int),
    "sdft_plan_launches": ([_P, ctypes.c_int], ctypes.c_int),
    "sdft_plan_describe": ([_P, ctypes.c_char_p, _I64], ctypes.c_int),
    "sdft_last_error": ([], ctypes.c_int),
    "sdft_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "sdft_version": ([], ctypes.c_char_p),
}

_lock = threading.Lock()
_lib = None


class SdftError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})" if what
                         else f"{status_string(status)} (status {status})")


def header_symbols() -> list[str]:
    """Names of every function include/sdft.h declares."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"SDFT_API[^;(]*?\b(sdft_\w+)\s*\(", text)))


def lib() -> ctypes.CDLL:
    """The loaded libsdft.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"libsdft.so not found at {LIB_PATH}; build it with "
                    "`python -m paper_2504_07264_gb300.build` (there is no CPU fallback)")
            handle = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                fn = getattr(handle, name)
                fn.argtypes = args
                fn.restype = res
            _lib = handle
        return _lib


# ---- thin C-named wrappers (marshalling only) ------------------------------
def sdft_plan_create(n: int, batch: int, dtype: int = SDFT_F32) -> int:
    return lib().sdft_plan_create(n, batch, dtype) or 0


def sdft_plan_create_ragged(lengths_ptr: int, count: int, dtype: int = SDFT_F32) -> int:
    return lib().sdft_plan_create_ragged(lengths_ptr, count, dtype) or 0


def sdft_plan_destroy(plan: int) -> None:
    lib().sdft_plan_destroy(plan)


def sdft_forward(plan, xr, xi, yr, yi, stream) -> int:
    return lib().sdft_forward(plan, xr, xi, yr, yi, stream)


def sdft_adjoint(plan, xr, xi, yr, yi, stream) -> int:
    return lib().sdft_adjoint(plan, xr, xi, yr, yi, stream)


def sdft_execute(plan, direction, xr, xi, yr, yi, stream) -> int:
    return lib().sdft_execute(plan, direction, xr, xi, yr, yi, stream)


def sdft_execute_host(plan, direction, xr, xi, yr, yi, stream) -> int:
    return lib().sdft_execute_host(plan, direction, xr, xi, yr, yi, stream)


def sdft_execute_noalloc(n, batch, direction, xr, xi, yr, yi, stream) -> int:
    return lib().sdft_execute_noalloc(n, batch, direction, xr, xi, yr, yi, stream)


def sdft_schedule_count(n: int, dtype: int = SDFT_F32) -> int:
    return lib().sdft_schedule_count(n, dtype)


def sdft_schedule_describe(n: int, dtype: int, index: int) -> str:
    need = lib().sdft_schedule_describe(n, dtype, index, None, 0)
    if need < 0:
        raise SdftError(-need, "sdft_schedule_describe")
    buf = ctypes.create_string_buffer(need + 1)
    lib().sdft_schedule_describe(n, dtype, index, buf, need + 1)
    return buf.value.decode()


def sdft_schedule_select(n: int, dtype: int, index: int) -> int:
    """Select compiled schedule `index` for later plans of (n, dtype).  The
    tuning table is applied first, so an explicit choice is never replaced
    by it afterwards."""
    from . import autotune
    autotune.ensure_applied()
    return lib().sdft_schedule_select(n, dtype, index)


def sdft_schedule_selected(n: int, dtype: int = SDFT_F32) -> int:
    return lib().sdft_schedule_selected(n, dtype)


def sdft_autotune(n, batch, dtype, xr, xi, yr, yi, reps, ms_out, stream) -> int:
    return lib().sdft_autotune(n, batch, dtype, xr, xi, yr, yi, reps, ms_out, stream)


def sdft_plan_set_host_mode(plan, mode: int) -> int:
    return lib().sdft_plan_set_host_mode(plan, mode)


def sdft_plan_set_grid(plan, grid: int) -> int:
    return lib().sdft_plan_set_grid(plan, grid)


def sdft_plan_grid(plan) -> int:
    return lib().sdft_plan_grid(plan)


def sdft_plan_set_wait_limit(plan, polls: int) -> int:
    return lib().sdft_plan_set_wait_limit(plan, polls)


def sdft_ragged_form_count(n: int) -> int:
    return lib().sdft_ragged_form_count(n)


def sdft_ragged_form_describe(n: int, form: int) -> str:
    need = lib().sdft_ragged_form_describe(n, form, None, 0)
    if need < 0:
        raise SdftError(-need, "sdft_ragged_form_describe")
    buf = ctypes.create_string_buffer(need + 1)
    lib().sdft_ragged_form_describe(n, form, buf, need + 1)
    return buf.value.decode()


def sdft_ragged_form_select(n: int, form: int) -> int:
    """Select form `form` of length n for work-queue plans created later.  The
    tuning table is applied first, so an explicit choice is never replaced by
    it afterwards."""
    from . import autotune
    autotune.ensure_applied()
    return lib().sdft_ragged_form_select(n, form)


def sdft_ragged_form_selected(n: int) -> int:
    return lib().sdft_ragged_form_selected(n)


def sdft_plan_set_ragged_form(plan, n: int, form: int) -> int:
    return lib().sdft_plan_set_ragged_form(plan, n, form)


def sdft_plan_ragged_form(plan, n: int) -> int:
    return lib().sdft_plan_ragged_form(plan, n)


def sdft_ragged_work_layout(lengths):
    """(phase_of, item_of, nitems) for a ragged batch of these lengths with the
    process-wide forms (host only; see include/sdft.h)."""
    import numpy as np
    arr = np.ascontiguousarray(lengths, dtype=np.int64)
    phase = np.empty(arr.size, dtype=np.int32)
    item = np.empty(arr.size, dtype=np.int32)
    nitems = np.zeros(4, dtype=np.int64)
    st = lib().sdft_ragged_work_layout(arr.ctypes.data, arr.size, phase.ctypes.data,
                                       item.ctypes.data, nitems.ctypes.data)
    if st != SDFT_OK:
        raise SdftError(st, "sdft_ragged_work_layout")
    return phase, item, nitems


def sdft_plan_ragged_autotune(plan, xr, xi, yr, yi, reps: int, stream) -> int:
    return lib().sdft_plan_ragged_autotune(plan, xr, xi, yr, yi, reps, stream)


def sdft_plan_inject_unreachable_wait(plan, on: int) -> int:
    return lib().sdft_plan_inject_unreachable_wait(plan, on)


def sdft_plan_sync_status(plan, stream) -> int:
    return lib().sdft_plan_sync_status(plan, stream)


def sdft_plan_n(plan) -> int:
    return lib().sdft_plan_n(plan)


def sdft_plan_batch(plan) -> int:
    return lib().sdft_plan_batch(plan)


def sdft_plan_points(plan) -> int:
    return lib().sdft_plan_points(plan)


def sdft_plan_dtype(plan) -> int:
    return lib().sdft_plan_dtype(plan)


def sdft_plan_launches(plan, direction: int = SDFT_FORWARD) -> int:
    return lib().sdft_plan_launches(plan, direction)


def sdft_plan_describe(plan) -> str:
    need = lib().sdft_plan_describe(plan, None, 0)
    if need < 0:
        raise SdftError(sdft_last_error(), "sdft_plan_describe")
    buf = ctypes.create_string_buffer(need + 1)
    lib().sdft_plan_describe(plan, buf, need + 1)
    return buf.value.decode()


def sdft_last_error() -> int:
    return lib().sdft_last_error()


def sdft_status_string(status: int) -> str:
    return lib().sdft_status_string(status).decode()


def sdft_version() -> str:
    return lib().sdft_version().decode()


status_string = sdft_status_string


# ---- torch-facing wrapper ---------------------------------------------------
def _check(status: int, what: str) -> None:
    if status != SDFT_OK:
        raise SdftError(status, what)


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Plan:
    """A plan for ``batch`` transforms of length ``n`` (or a ragged batch).

    ``forward``/``adjoint`` take float32 CUDA tensors of shape (batch, n) (or
    flat tensors of the plan's total length for ragged plans) and run on the
    current torch stream unless ``stream`` is given.
    """

    def __init__(self, n: int | None = None, batch: int | None = None, dtype: int = SDFT_F32,
                 lengths=None):
        self._h = 0
        from . import autotune
        autotune.ensure_applied()
        if lengths is not None:
            import numpy as np
            arr = np.ascontiguousarray(lengths, dtype=np.int64)
            h = sdft_plan_create_ragged(arr.ctypes.data, arr.size, dtype)
            self.lengths = arr.copy()
        else:
            h = sdft_plan_create(int(n), int(batch), dtype)
            self.lengths = None
        if not h:
            raise SdftError(sdft_last_error(), "sdft_plan_create")
        self._h = h
        self.n = sdft_plan_n(h)
        self.batch = sdft_plan_batch(h)
        self.points = sdft_plan_points(h)
        self.dtype = dtype

    @property
    def handle(self) -> int:
        if not self._h:
            raise SdftError(SDFT_ERR_BAD_PLAN, "plan already destroyed")
        return self._h

    def describe(self) -> str:
        return sdft_plan_describe(self.handle)

    def launches(self, direction: int = SDFT_FORWARD) -> int:
        return sdft_plan_launches(self.handle, direction)

    def destroy(self) -> None:
        if self._h:
            sdft_plan_destroy(self._h)
            self._h = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def _shape_ok(self, t) -> bool:
        return t.numel() == self.points

    def execute(self, direction: int, xr, xi, yr=None, yi=None, stream=None):
        import torch
        for name, t in (("xr", xr), ("xi", xi)):
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() \
                    or not self._shape_ok(t):
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of "
                                 f"{self.points} elements, got {tuple(t.shape)} {t.dtype}")
        if yr is None:
            yr = torch.empty_like(xr)
        if yi is None:
            yi = torch.empty_like(xi)
        for name, t in (("yr", yr), ("yi", yi)):
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() \
                    or not self._shape_ok(t):
                raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of "
                                 f"{self.points} elements")
        st = sdft_execute(self.handle, direction, xr.data_ptr(), xi.data_ptr(), yr.data_ptr(),
                          yi.data_ptr(), _stream_handle(stream))
        _check(st, "sdft_forward" if direction == SDFT_FORWARD else "sdft_adjoint")
        return yr, yi

    def forward(self, xr, xi, yr=None, yi=None, stream=None):
        return self.execute(SDFT_FORWARD, xr, xi, yr, yi, stream)

    def adjoint(self, xr, xi, yr=None, yi=None, stream=None):
        return self.execute(SDFT_ADJOINT, xr, xi, yr, yi, stream)

    def execute_host(self, direction: int, xr, xi, yr, yi, stream=None) -> None:
        """Host arrays (numpy float32, C-contiguous, or pinned CPU tensors)."""
        ptrs = []
        for a in (xr, xi, yr, yi):
            if hasattr(a, "data_ptr"):
                if a.is_cuda or not a.is_contiguous() or a.numel() != self.points:
                    raise ValueError("host tensors must be contiguous CPU tensors of the plan size")
                ptrs.append(a.data_ptr())
            else:
                if a.dtype.name != "float32" or not a.flags["C_CONTIGUOUS"] or a.size != self.points:
                    raise ValueError("host arrays must be C-contiguous float32 of the plan size")
                ptrs.append(a.ctypes.data)
        st = sdft_execute_host(self.handle, direction, *ptrs, _stream_handle(stream))
        _check(st, "sdft_execute_host")

    @property
    def grid(self) -> int:
        return sdft_plan_grid(self.handle)

    def set_grid(self, grid: int) -> None:
        _check(sdft_plan_set_grid(self.handle, grid), "sdft_plan_set_grid")

    def set_host_mode(self, mode: int) -> None:
        _check(sdft_plan_set_host_mode(self.handle, mode), "sdft_plan_set_host_mode")

    def ragged_form(self, n: int) -> int:
        """Work-queue plans: the form length n runs in."""
        v = sdft_plan_ragged_form(self.handle, n)
        if v < 0:
            raise SdftError(-v, "sdft_plan_ragged_form")
        return v

    def set_ragged_form(self, n: int, form: int) -> None:
        _check(sdft_plan_set_ragged_form(self.handle, n, form), "sdft_plan_set_ragged_form")

    def ragged_autotune(self, xr, xi, yr, yi, reps: int = 10, stream=None) -> int:
        """Time each length's forms on these device tensors (the plan's
        layout), one length at a time, longest first, and keep the fastest;
        returns the mask of lengths (bit log2 N) left on a form other than 0."""
        v = sdft_plan_ragged_autotune(self.handle, xr.data_ptr(), xi.data_ptr(), yr.data_ptr(),
                                      yi.data_ptr(), reps, _stream_handle(stream))
        if v < 0:
            raise SdftError(-v, "sdft_plan_ragged_autotune")
        return v

    def sync_status(self, stream=None) -> int:
        return sdft_plan_sync_status(self.handle, _stream_handle(stream))
