// split.h -- internal interface of the split-precision tensor-core kernels.
#pragma once

#include "launch.h"

namespace sdft {

struct SplitInfo {
    KernelInfo kern;                                   // launch, tables, occupancy
    size_t aux_bytes;                                  // block-matrix images (device)
    cudaError_t (*make_aux)(void* dst, cudaStream_t);  // fills them
};

// log2 N in {8, 10}, dtype SDFT_F32_SPLIT_BF16 or SDFT_F32_SPLIT_FP16; else null.
const SplitInfo* split_kernel(int logn, int dtype);

}  // namespace sdft
