// ragged.h -- internal interface of the persistent work-queue kernel
// (ragged.cu): ragged batches, and uniform batches of long transforms.
#pragma once

#include "launch.h"

namespace sdft {

// The kernel runs as thread-block clusters of kRaggedCluster CTAs of 128
// threads (three CTAs per SM).  Every length class runs one of its compiled
// *forms* (a routine: radix split, values per thread, CTAs per transform,
// transforms per tile).  A form holds a transform in the shared memory of
// q = 8, 4 or 2 CTAs (a group of the cluster: ranks g*q .. g*q+q-1) or runs
// a tile of transforms in one CTA (q = 1).  The work is split into four
// phases by q; a cluster runs the q = 8 phase as one group, then splits into
// two groups of four, then into pairs, then into single CTAs:
//   phase 0..2 (q = 8, 4, 2): one item per transform, {routine, row start lo,
//                             row start hi, N}, taken by the groups in turn; the
//                             groups of a cluster share its barriers
//   phase 3    (q = 1)      : row items {routine, first transform in the row
//                             order, count, 0}, claimed by each CTA
constexpr int kRaggedCluster = 8;
constexpr int kRaggedPhases = 4;
constexpr int kRaggedRoutines = 48;      // routine codes 0 .. kRaggedRoutines - 1

inline int ragged_phase_of(int q) { return q == 8 ? 0 : q == 4 ? 1 : q == 2 ? 2 : 3; }

// Kernel arguments, passed by value.
struct RaggedArgs {
    const float* xr;
    const float* xi;
    float* yr;
    float* yi;
    const int4* items[kRaggedPhases];   // each phase's items, in claim order
    int nitems[kRaggedPhases];
    const long long* offsets;           // row items: row start (floats) of each transform
    int* counters;                      // [kRaggedPhases] claim counters (only the row phase
                                        // claims), then a word that stays zero (all zeroed
                                        // before each launch)
    int* status;                        // plan status word (SDFT_ERR_TIMEOUT on a wait that gave up)
    int wait_polls;                     // bound of every wait (polls)
    int inject;                         // tests: every group item first waits for a word nothing sets
    const float2* tw[kRaggedRoutines];  // twiddle tables of each routine
    W64 w;
};

// One compiled routine of the work-queue kernel.
struct RaggedForm {
    const char* name;
    int code;                   // routine code (the item's first word)
    int logn;
    int q;                      // CTAs per transform (8, 4, 2), or 1: a tile of one CTA
    int per_item;               // q = 1: transforms per tile
    int ntables;
    TableDesc tables[4];
    int64_t tw_entries;
};

int ragged_form_count(int logn);                 // log2 N in [2, 16], else 0
const RaggedForm* ragged_form(int logn, int f);  // null past the last
int ragged_threads();
size_t ragged_smem();
const void* ragged_kernel_fn(bool adj);
cudaError_t ragged_prepare();
int ragged_resident_ctas();                      // whole clusters resident over the GPU

}  // namespace sdft
