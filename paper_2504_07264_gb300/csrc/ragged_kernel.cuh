// ragged_kernel.cuh -- the persistent work-queue kernel for ragged batches
// (its routines, routine codes and phases), compiled once per direction
// (ragged_fwd.cu, ragged_adj.cu); ragged.cu holds the host side.
//
// One persistent launch for a batch of mixed power-of-two lengths.
//
// The kernel runs as thread-block clusters of 8 CTAs of 128 threads, three
// CTAs per SM.  The plan gives every length class one of its compiled forms
// (ragged.h) and orders the work into four phases by the number of CTAs a
// transform occupies:
//   phase 0: transforms held by the whole cluster (N = 65536, or N = 32768 on
//            eight CTAs of 4096 points),
//   phase 1: transforms held by four CTAs, phase 2: by two -- the cluster passes
//            of kernels_cluster.cuh, the intermediate in distributed shared
//            memory,
//   phase 3: row tiles of one CTA (transforms of up to 8192 points).
// A cluster runs phase 0 as one group, then splits into two groups of four,
// then into four pairs, then into single CTAs.  In a group phase the grid's
// groups take the phase's transforms in turn (group g: items g, g + G, ...),
// which needs no claims because the items of a class cost the same, and lets
// every CTA bring its share of the group's next transform into L2 a whole item
// ahead; the PER = 8 / q transforms a cluster holds at a time share the
// hardware cluster barrier (a group without a transform in the last round
// takes the barriers only).  Row tiles, of very different sizes, are claimed
// one at a time by each CTA with an atomicAdd (the next claim is made while
// the current tile runs), so CTAs that finish their groups early take more of
// them.  (Groups synchronising alone through mbarriers measured no faster and
// doubled the kernel's code, which the instruction cache pays for.)
//
// A transform is computed with the same arithmetic and tables as the uniform
// kernel of the same form.  The row-tile claim counter is zeroed by a memset
// node that precedes the kernel in the plan's CUDA graph.  Every wait is bounded:
// past its limit it records SDFT_ERR_TIMEOUT in the plan's status word, and
// once the word is set no wait blocks any more.  The only such wait is the
// testing hook: a plan can make every group item first wait for a word that
// nothing sets.
#pragma once

#include "../../include/sdft.h"
#include "kernels_cluster.cuh"
#include "kernels_rows.cuh"
#include "ragged.h"

namespace sdft {
namespace rq {

constexpr int kThreads = 128;
constexpr int kMinBlocks = 3;

// Row routines: one CTA of 128 threads runs a tile of G transforms.
//                LOGN LOGE LR0 LR1 LR2   G  SBX MINB DIT
using R2 = RowCfg<2, 2, 2, 0, 0, 128>;
using R3 = RowCfg<3, 3, 3, 0, 0, 128>;
using R4 = RowCfg<4, 4, 4, 0, 0, 128>;
using R5 = RowCfg<5, 5, 5, 0, 0, 128>;
using R6 = RowCfg<6, 3, 3, 3, 0, 16, 2>;
using R7 = RowCfg<7, 4, 4, 3, 0, 16>;
using R8 = RowCfg<8, 4, 4, 4, 0, 8>;
using R8b = RowCfg<8, 5, 5, 3, 0, 16, 8>;           // 8 threads x 32 values, radix [32,8]
using R9 = RowCfg<9, 5, 5, 4, 0, 8, 16>;
using R9b = RowCfg<9, 4, 4, 4, 1, 4>;               // 32 threads, radix [16,16,2]
using R10 = RowCfg<10, 5, 5, 5, 0, 4>;
using R10b = RowCfg<10, 4, 4, 3, 3, 2>;             // 64 threads, radix [16,8,8]
using R11 = RowCfg<11, 5, 5, 4, 2, 2>;              // 64 threads, radix [32,16,4]
using R11b = RowCfg<11, 4, 4, 4, 3, 1>;             // 128 threads, radix [16,16,8]
using R12 = RowCfg<12, 5, 5, 5, 2, 1, 0, 1, false, true>;   // 128 threads, radix [32,32,4], swizzled exchange

// routine codes (the first word of every work item)
enum : int {
    kR2, kR3, kR4, kR5, kR6, kR7, kR8, kR8b, kR9, kR9b, kR10, kR10b, kR11, kR11b, kR12,
    kC13, kC14q, kC15q, kC16e, kRoutineCount
};
static_assert(kRoutineCount <= kRaggedRoutines, "routine table");

constexpr size_t smax(size_t a, size_t b) { return a > b ? a : b; }

// The kernel declares no static shared memory: its dynamic buffer then starts
// on the CTA's shared-memory window itself, so the Y arrays of the cluster
// forms are 128-byte aligned and every pass-2 warp load of a peer's Y is one
// whole line (one network transaction; with a few bytes of static shared
// memory in front, each would straddle two lines).  The CTA's small state
// sits in a tail after the data region.
struct RaggedTail {
    int4 work[2];          // row tiles: this CTA's claimed records
    int4 next[2];          // group phases: the group's next item, alternating slots
    int ok;                // outcome of a bounded wait, for the whole CTA
};
// Every routine fits in 64 KiB: three CTAs of 64 KiB (plus the 1 KiB the
// runtime reserves per CTA and the 128-byte tail) stay within the 196 KiB
// shared-memory carveout, which leaves 60 KiB of L1 for the rotation tables
// and the input lines; 2 KiB more per CTA forces the 228 KiB carveout, halves
// L1 and cost 15 % at N = 65536.  (A transform of 8192 points runs on two
// CTAs: a one-CTA tile of it, 128 threads x 64 values with an XOR-swizzled
// exchange of exactly 64 KiB, measured 145 against 152 Gpts/s.)
constexpr size_t kData = smax(
    smax(smax(R9::SMEM, R10::SMEM), smax(smax(R10b::SMEM, R11::SMEM), smax(R11b::SMEM, R12::SMEM))),
    smax(smax(Cluster13::SMEM, Cluster14q::SMEM), smax(Cluster15q::SMEM, Cluster16e::SMEM)));
static_assert(kData <= 64 * 1024, "three CTAs per SM within the 196 KiB carveout");
constexpr size_t kSmem = kData + ((sizeof(RaggedTail) + 127) / 128) * 128;
static_assert(kData % 128 == 0, "the tail starts 128-byte aligned");

__device__ __forceinline__ RaggedTail* tail_of(float* smem) {
    return reinterpret_cast<RaggedTail*>(reinterpret_cast<char*>(smem) + kData);
}

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Thread 0 waits (bounded) until *word >= target; the CTA learns the outcome.
// false: the wait gave up now or an earlier one did (status already set).
__device__ __forceinline__ bool cta_wait(const int* word, int target, const RaggedArgs& a,
                                         int& s_ok) {
    if (threadIdx.x == 0) {
        int ok = 0;
        if (ld_acquire(a.status) == 0) {
            for (int i = 0; i < a.wait_polls; ++i) {
                if (ld_acquire(word) >= target) { ok = 1; break; }
                if ((i & 1023) == 1023 && ld_acquire(a.status) != 0) break;
                __nanosleep(128);
            }
            if (!ok) atomicCAS(a.status, 0, SDFT_ERR_TIMEOUT);
        }
        s_ok = ok;
    }
    __syncthreads();
    const bool ok = s_ok != 0;
    __syncthreads();
    return ok;
}

// the record that ends a phase
__device__ __forceinline__ int4 end_record() { return make_int4(-1, 0, 0, 0); }

__device__ __forceinline__ int4 load_item(const RaggedArgs& a, const int phase, const int i) {
    return i < a.nitems[phase] ? a.items[phase][i] : end_record();
}

// One transform of form CFG (CFG::Q CTAs, this one at position q of the group
// starting at cluster rank g0); rec = {routine, row start lo, row start hi, N}.
template <class CFG, bool ADJ, class MID, class BARA, class RD>
__device__ __forceinline__ void group_item(const RaggedArgs& a, const int4 rec, float* smem,
                                           const uint32_t q, const uint32_t g0, const MID& mid,
                                           const BARA& bar_a, const RD& rd) {
    constexpr int A = CFG::A, C = CFG::C;
    static_assert(CFG::THREADS == kThreads && CFG::SMEM <= kData, "group routine shape");
    const int tid = (int)threadIdx.x;
    if (a.inject) cta_wait(a.counters + kRaggedPhases, 1, a, tail_of(smem)->ok);
    const long long off = (long long)(((uint64_t)(uint32_t)rec.z << 32) | (uint32_t)rec.y);
    const float2* tw = a.tw[rec.x];
    const int col = (int)q * CFG::CQ + tid % CFG::CQ;
    const int d = (int)q * CFG::AQ + tid % CFG::AQ;
    // the input is read only (the C ABI forbids partial overlap with the
    // output, and in place each element is read before it is written), so it
    // is loaded through the read-only data path
    const float* __restrict__ gxr = a.xr + off;
    const float* __restrict__ gxi = a.xi + off;
    auto ld = [&](int L, float& r, float& i) {
        r = __ldg(gxr + col + C * L);
        i = __ldg(gxi + col + C * L);
    };
    pass1<CFG, ADJ>(ld, mid, smem, tid, col, tw, a.w);
    bar_a();
    float* const gyr = a.yr + off;
    float* const gyi = a.yi + off;
    auto st = [&](int k2, float r, float i) {
        __stcs(gyr + d + A * k2, r);   // evict-first: keeps L2 for the prefetched input
        __stcs(gyi + d + A * k2, i);
    };
    pass2<CFG, ADJ>(st, smem, (uint32_t)__cvta_generic_to_shared(smem), tid, d, g0, tw, a.w, rd);
}

// Phase PHASE: the grid's groups of Q CTAs take the phase's transforms in
// turn (group g: items g, g + G, g + 2G, ..., G groups), all of equal size
// within a class, so no claims are needed; at the top of each item every CTA
// brings its share of the group's next transform into L2.
template <int Q, int PHASE, bool ADJ>
__device__ __forceinline__ void group_phase(const RaggedArgs& a, float* smem, const uint32_t rank) {
    static_assert(Q == (kRaggedCluster >> PHASE), "a phase's groups hold its routines' transforms");
    constexpr int PER = kRaggedCluster / Q;   // groups per cluster
    const uint32_t g0 = rank & ~(uint32_t)(Q - 1), q = rank & (uint32_t)(Q - 1);
    const int sub = (int)(rank / Q);
    const int stride = (int)(gridDim.x / kRaggedCluster) * PER;   // groups in the grid
    auto sync = [] {
        cluster_arrive();
        cluster_wait();
    };
    const ClusterReadsDone rd{};
    // Thread 0 issues the load of the group's next item at the top of the
    // current one and, between the two register steps of pass 1 (once it has
    // arrived), stores it into a slot of the CTA's tail and starts the L2
    // prefetch of this CTA's share of that transform; the CTA reads the slot
    // at the end of the item, so no item starts with a dependent global load.
    // Two slots alternate: a slot is rewritten only after the CTA barriers of
    // the item that read it.
    RaggedTail* const tl = tail_of(smem);
    int base = (int)cluster_id() * PER;   // the cluster's first item of this round
    int par = 0;
    int4 rec = load_item(a, PHASE, base + sub);
    while (base < a.nitems[PHASE]) {      // the same number of rounds for every CTA of a cluster
        base += stride;
        int4 nxt = end_record();
        if (threadIdx.x == 0) nxt = load_item(a, PHASE, base + sub);
        auto mid = [&] {
            if (threadIdx.x == 0) {
                tl->next[par] = nxt;
                if (nxt.x >= 0) {
                    const long long noff =
                        (long long)(((uint64_t)(uint32_t)nxt.z << 32) | (uint32_t)nxt.y);
                    const long long share = nxt.w / Q;
                    prefetch_l2(a.xr + noff + q * share, (uint32_t)(share * 4));
                    prefetch_l2(a.xi + noff + q * share, (uint32_t)(share * 4));
                }
            }
        };
        switch (rec.x) {
            case kC16e: if constexpr (Q == 8) group_item<Cluster16e, ADJ>(a, rec, smem, q, g0, mid, sync, rd); break;
            case kC15q: if constexpr (Q == 8) group_item<Cluster15q, ADJ>(a, rec, smem, q, g0, mid, sync, rd); break;
            case kC14q: if constexpr (Q == 4) group_item<Cluster14q, ADJ>(a, rec, smem, q, g0, mid, sync, rd); break;
            case kC13: if constexpr (Q == 2) group_item<Cluster13, ADJ>(a, rec, smem, q, g0, mid, sync, rd); break;
            default:   // no transform for this group in this round: the barriers only
                if (threadIdx.x == 0) tl->next[par] = nxt;
                sync();
                sync();
                break;
        }
        rec = tl->next[par];
        par ^= 1;
    }
}

template <class CFG, bool ADJ>
__device__ __forceinline__ void row_tile(const RaggedArgs& a, const int4 item, float* smem) {
    using S = typename CFG::S;
    static_assert(CFG::THREADS == kThreads, "row routines use the kernel's 128 threads");
    static_assert(CFG::SMEM <= kData, "row routine exceeds the kernel's shared memory");
    const int t = (int)threadIdx.x & (S::T - 1);
    const int g = (int)threadIdx.x >> S::LOGT;
    const bool active = g < item.z;
    const long long row = active ? a.offsets[item.y + g] : 0;
    float* const s_re = smem + g * CFG::BUF;
    float* const s_im = s_re + CFG::PLANE;
    rows_tile<CFG, ADJ>(a.xr + row, a.xi + row, a.yr + row, a.yi + row, active, t, s_re, s_im,
                        a.tw[item.x], a.w);
}

// Phase 3: every CTA claims row tiles on its own.
template <bool ADJ>
__device__ __forceinline__ void row_phase(const RaggedArgs& a, float* smem, int4* slots) {
    constexpr int P = kRaggedPhases - 1;
    if (threadIdx.x == 0) slots[0] = load_item(a, P, atomicAdd(a.counters + P, 1));
    __syncthreads();
    for (int par = 0;; par ^= 1) {
        const int4 rec = slots[par];
        if (rec.x < 0) break;
        int claim = 0;
        if (threadIdx.x == 0) claim = atomicAdd(a.counters + P, 1);
        switch (rec.x) {
            case kR2: row_tile<R2, ADJ>(a, rec, smem); break;
            case kR3: row_tile<R3, ADJ>(a, rec, smem); break;
            case kR4: row_tile<R4, ADJ>(a, rec, smem); break;
            case kR5: row_tile<R5, ADJ>(a, rec, smem); break;
            case kR6: row_tile<R6, ADJ>(a, rec, smem); break;
            case kR7: row_tile<R7, ADJ>(a, rec, smem); break;
            case kR8: row_tile<R8, ADJ>(a, rec, smem); break;
            case kR8b: row_tile<R8b, ADJ>(a, rec, smem); break;
            case kR9: row_tile<R9, ADJ>(a, rec, smem); break;
            case kR9b: row_tile<R9b, ADJ>(a, rec, smem); break;
            case kR10: row_tile<R10, ADJ>(a, rec, smem); break;
            case kR10b: row_tile<R10b, ADJ>(a, rec, smem); break;
            case kR11: row_tile<R11, ADJ>(a, rec, smem); break;
            case kR11b: row_tile<R11b, ADJ>(a, rec, smem); break;
            case kR12: row_tile<R12, ADJ>(a, rec, smem); break;
            default: break;
        }
        if (threadIdx.x == 0) slots[par ^ 1] = load_item(a, P, claim);
        __syncthreads();   // the slot, and shared memory before the next tile
    }
}

template <bool ADJ>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_ragged(const RaggedArgs a) {
    extern __shared__ __align__(128) float4 smem4[];
    float* const smem = reinterpret_cast<float*>(smem4);
    int4* const s_work = tail_of(smem)->work;
    const uint32_t rank = cluster_ctarank();
    // every CTA of the cluster is running before any of its shared memory is
    // accessed from another CTA
    cluster_arrive();
    cluster_wait();
    if (a.nitems[0] > 0) group_phase<8, 0, ADJ>(a, smem, rank);
    if (a.nitems[1] > 0) group_phase<4, 1, ADJ>(a, smem, rank);
    if (a.nitems[2] > 0) group_phase<2, 2, ADJ>(a, smem, rank);
    if (a.nitems[3] > 0) row_phase<ADJ>(a, smem, s_work);
    // No CTA exits while another CTA of its cluster may still read its shared
    // memory (the row phase is local, but a CTA whose group phases ended
    // early must outlive its peers' last remote reads).
    cluster_arrive();
    cluster_wait();
}

}  // namespace rq
}  // namespace sdft
