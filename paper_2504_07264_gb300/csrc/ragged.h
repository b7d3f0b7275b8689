// ragged.h -- internal interface of the persistent work-queue kernel
// (ragged.cu): ragged batches, and uniform batches of long transforms.
#pragma once

#include "launch.h"

namespace sdft {

// item.x: log2 N for row items; kPass1 + log2 N / kPass2 + log2 N for the two
// passes of a long transform.
constexpr int kPass1 = 100;
constexpr int kPass2 = 200;

// Kernel arguments, passed by value.
struct RaggedArgs {
    const float* xr;
    const float* xi;
    float* yr;
    float* yi;
    const long long* offsets;       // row items: row start (floats) of each transform, in work order
    const int4* items;              // (kind, first transform / long index, count / tile, dependency)
    int nitems;
    int* counter;                   // work counter, zero at launch
    const long long* long_offsets;  // long transforms: row start (floats)
    const int* long_slot;           // long transforms: scratch slot
    const int* tiles2;              // long transforms: number of pass-2 items
    int* done1;                     // long transforms: finished pass-1 items (zero at launch)
    int* done2;                     // long transforms: finished pass-2 items (zero at launch)
    int* status;                    // plan status word (SDFT_ERR_TIMEOUT on a wait that gave up)
    int wait_polls;                 // bound of every wait (polls of ~128 ns)
    int dep_extra;                  // added to every pass-2 wait target (0; tests set 1 to
                                    // make the dependency unreachable)
    long long slot_size;            // float2 entries per scratch slot
    float2* scratch;                // slots
    const float2* tw[17];           // twiddle tables of each length class (by log2 N)
    W64 w;
};

// One length class of the work-queue kernel.
struct RaggedClass {
    int logn;
    int per_item;               // transforms per row item (1 for long classes)
    bool large;                 // split into pass-1 / pass-2 items
    int tiles1, tiles2;         // items per pass of one long transform
    int ntables;
    TableDesc tables[4];
    int64_t tw_entries;
};

const RaggedClass* ragged_class(int logn);   // log2 N in [2, 16], else null
int ragged_threads();
size_t ragged_smem();
int64_t ragged_slot_size();                  // float2 entries per scratch slot
const void* ragged_kernel_fn(bool adj);
cudaError_t ragged_prepare();
int ragged_blocks_per_sm();

}  // namespace sdft
