"""Planar split-complex DFT for NVIDIA GB300 (sm_103a).

The batched complex DFT of Eq. (1) computed with real and imaginary parts
kept in separate float32 planes (Cariow, arXiv 2504.07264).  The compute path
is the CUDA library libsdft.so (C ABI in include/sdft.h); this package holds
its Python binding and a torch.autograd.Function on top.  Build the library
with ``python -m paper_2504_07264_gb300.build``.
"""
from .sdft import (SDFT_ADJOINT, SDFT_F32, SDFT_F32_SPLIT_BF16,  # noqa: F401
                   SDFT_F32_SPLIT_FP16, SDFT_FORWARD, Plan, SdftError)


def __getattr__(name):
    # torch-dependent helpers load lazily so the ctypes binding imports without torch
    if name in ("split_dft", "split_dft_adjoint", "SplitDFT", "SplitDFTAdjoint", "get_plan",
                "clear_plan_cache"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
