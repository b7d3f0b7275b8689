// ragged_fwd.cu -- the forward instance of the work-queue kernel (ragged_kernel.cuh),
// in a translation unit of its own so that the two directions compile in parallel.
#include "ragged_kernel.cuh"

namespace sdft {

const void* ragged_kernel_fwd() { return reinterpret_cast<const void*>(rq::k_ragged<false>); }

}  // namespace sdft
