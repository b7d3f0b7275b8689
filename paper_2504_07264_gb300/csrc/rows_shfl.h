// rows_shfl.h -- short transforms spread over a few lanes of a warp, with
// butterflies across lanes by __shfl_xor_sync (rows_shfl.cu).
#pragma once

#include "launch.h"

namespace sdft {

// idx-th shuffle candidate for length 2^logn (N = 16 .. 64), or null.
const KernelInfo* rows_shfl_candidate(int logn, int idx);

}  // namespace sdft
