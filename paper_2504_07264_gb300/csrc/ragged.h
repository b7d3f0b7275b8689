// ragged.h -- internal interface of the ragged persistent kernel (ragged.cu).
#pragma once

#include "launch.h"

namespace sdft {

// Kernel arguments, passed by value.
struct RaggedArgs {
    const float* xr;
    const float* xi;
    float* yr;
    float* yi;
    const long long* offsets;   // row start (in floats) of each transform, in work order
    const int4* items;          // work items: (log2 N, first transform, count, 0)
    int nitems;
    int* counter;               // work counter, zero at launch
    float2* scratch;            // one 65536-point slot per CTA (classes N >= 32768)
    const float2* tw[17];       // twiddle tables of each length class (by log2 N)
    W64 w;
};

// One length class of the ragged kernel.
struct RaggedClass {
    int logn;
    int per_item;               // transforms per work item
    bool large;                 // two-pass class (needs scratch)
    int ntables;
    TableDesc tables[4];
    int64_t tw_entries;
};

const RaggedClass* ragged_class(int logn);   // log2 N in [2, 16], else null
int ragged_threads();
size_t ragged_smem();
int64_t ragged_scratch_per_cta();            // float2 entries
const void* ragged_kernel_fn(bool adj);
cudaError_t ragged_prepare();
int ragged_blocks_per_sm();

}  // namespace sdft
