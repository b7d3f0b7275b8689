// ragged.h -- internal interface of the persistent work-queue kernel
// (ragged.cu): ragged batches, and uniform batches of long transforms.
#pragma once

#include "launch.h"

namespace sdft {

// The kernel runs as thread-block clusters of kRaggedCluster CTAs.  A cluster
// claims one cluster item at a time:
//   x = log2 N (2 .. 13): a group of up to 8 row items; CTA r of the cluster
//       runs row item y + r if r < z
//   x = kLong + log2 N (14 .. 16): long transforms y .. y + z - 1 of the long
//       list, one per N / 8192 CTAs of the cluster (z <= 8 * 8192 / N)
// A row item (x = log2 N, y = first transform in the row order, z = count)
// is `per_item` transforms of one length run by one CTA.
constexpr int kLong = 100;
constexpr int kRaggedCluster = 8;

// Kernel arguments, passed by value.
struct RaggedArgs {
    const float* xr;
    const float* xi;
    float* yr;
    float* yi;
    const long long* offsets;       // row items: row start (floats) of each transform, in work order
    const int4* items;              // row items
    const int4* citems;             // cluster items
    int nitems;                     // cluster items
    int* counter;                   // claimed cluster items (zero at launch)
    const long long* long_offsets;  // long transforms: row start (floats)
    int* never;                     // a word that stays zero (target of injected waits)
    int* status;                    // plan status word (SDFT_ERR_TIMEOUT on a wait that gave up)
    int wait_polls;                 // bound of every wait (polls of ~128 ns)
    int inject;                     // tests: every long item first waits for `never` to become 1
    unsigned alt;                   // bit l: class log2 N = l uses its alternative routine
    const float2* tw[17];           // twiddle tables of each length class (by log2 N)
    W64 w;
};

// One length class of the work-queue kernel.
struct RaggedClass {
    int logn;
    int per_item;               // transforms per row item, or per cluster item (long classes)
    bool large;                 // a long class: cluster items
    int ntables;
    TableDesc tables[4];
    int64_t tw_entries;
};

const RaggedClass* ragged_class(int logn);   // log2 N in [2, 16], else null
int ragged_threads();
size_t ragged_smem();
const void* ragged_kernel_fn(bool adj);
cudaError_t ragged_prepare();
int ragged_resident_ctas();                  // whole clusters resident over the GPU
unsigned ragged_alt_classes();               // bit l: class l has an alternative routine

}  // namespace sdft
