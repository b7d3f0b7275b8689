// ragged_adj.cu -- the adjoint instance of the work-queue kernel (ragged_kernel.cuh),
// in a translation unit of its own so that the two directions compile in parallel.
#include "ragged_kernel.cuh"

namespace sdft {

const void* ragged_kernel_adj() { return reinterpret_cast<const void*>(rq::k_ragged<true>); }

}  // namespace sdft
