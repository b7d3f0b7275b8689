"""CPU oracle for the split complex DFT (test infrastructure only).

Only tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package; the CUDA library never does.
"""
from .oracle import (adjoint_direct, adjoint_factored, build, dft_direct,  # noqa: F401
                     dft_direct_bins, dft_factored_dif, dft_factored_dit, dit_stages,
                     thread_count)
