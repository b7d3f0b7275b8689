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
// then into four pairs, then into single CTAs; groups never merge again and
// synchronise only their own CTAs: the whole cluster with the hardware cluster
// barrier, smaller groups with mbarriers that each CTA of the group arrives on
// remotely (one thread per CTA, release at cluster scope; the polling thread
// acquires, then releases its CTA with a CTA barrier).  Transforms that share
// a cluster do not wait for each other.
//
// Work: in a group phase the grid's groups take the phase's transforms in turn
// (group g: items g, g + G, ...), which needs no claims because the items of a
// class cost the same, and lets every CTA bring its share of the group's next
// transform into L2 a whole item ahead.  Row tiles, of very different sizes,
// are claimed one at a time by each CTA with an atomicAdd (the next claim is
// made while the current tile runs); early groups thereby take more of them.
//
// A transform is computed with the same arithmetic and tables as the uniform
// kernel of the same form.  The row-tile claim counter is zeroed by a memset
// node that precedes the kernel in the plan's CUDA graph.  Every wait is bounded:
// past its limit it records SDFT_ERR_TIMEOUT in the plan's status word, and
// once the word is set no wait blocks any more (the results of that launch are
// undefined, but every access stays within the plan's buffers and every CTA
// keeps its shared memory until its cluster ends).  For tests, a plan can make
// every group item first wait for a word that nothing sets.
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
using R5D = RowCfg<5, 5, 5, 0, 0, 128, 0, 1, true>;
using R6 = RowCfg<6, 3, 3, 3, 0, 16, 2>;
using R6D = RowCfg<6, 3, 3, 3, 0, 16, 2, 1, true>;
using R7 = RowCfg<7, 4, 4, 3, 0, 16>;
using R7D = RowCfg<7, 4, 4, 3, 0, 16, 0, 1, true>;
using R8 = RowCfg<8, 4, 4, 4, 0, 8>;
using R8D = RowCfg<8, 4, 4, 4, 0, 8, 0, 1, true>;
using R8b = RowCfg<8, 5, 5, 3, 0, 16, 8>;           // 8 threads x 32 values, radix [32,8]
using R9 = RowCfg<9, 5, 5, 4, 0, 8, 16>;
using R9D = RowCfg<9, 5, 5, 4, 0, 8, 16, 1, true>;
using R9b = RowCfg<9, 4, 4, 4, 1, 4>;               // 32 threads, radix [16,16,2]
using R10 = RowCfg<10, 5, 5, 5, 0, 4>;
using R10D = RowCfg<10, 5, 5, 5, 0, 4, 0, 1, true>;
using R11 = RowCfg<11, 5, 5, 4, 2, 2>;              // 64 threads, radix [32,16,4]
using R12 = RowCfg<12, 5, 5, 5, 2, 1>;              // 128 threads, radix [32,32,4]

// routine codes (the first word of every work item)
enum : int {
    kR2, kR3, kR4, kR5, kR5D, kR6, kR6D, kR7, kR7D, kR8, kR8D, kR8b, kR9, kR9D, kR9b,
    kR10, kR10D, kR11, kR12,
    kC13, kC14e, kC14q, kC15e, kC15q, kC16e, kRoutineCount
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
    uint64_t bar[2][2];    // mbarriers of the groups of 4 and of 2: [A, B]
    int ok;                // outcome of a bounded wait, for the whole CTA
};
// Every routine fits in 64 KiB: three CTAs of 64 KiB (plus the 1 KiB the
// runtime reserves per CTA and the 128-byte tail) stay within the 196 KiB
// shared-memory carveout, which leaves 60 KiB of L1 for the rotation tables
// and the input lines; 2 KiB more per CTA forces the 228 KiB carveout, halves
// L1 and cost 15 % at N = 65536 (a transform of 8192 points therefore runs on
// two CTAs rather than as a row tile).
constexpr size_t kData = smax(
    smax(smax(R9::SMEM, R10::SMEM), smax(R11::SMEM, R12::SMEM)),
    smax(smax(smax(Cluster13::SMEM, Cluster14e::SMEM), smax(Cluster14q::SMEM, Cluster15e::SMEM)),
         smax(Cluster15q::SMEM, Cluster16e::SMEM)));
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
// the status word, read without ordering anything (an acquire at GPU scope
// would also discard this SM's L1 lines, the rotation tables among them)
__device__ __forceinline__ int ld_status(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
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

__device__ __forceinline__ void mbar_init(uint32_t addr, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(addr), "r"(count) : "memory");
}
// One arrival on the mbarrier at `cluster_addr` (any CTA of the cluster),
// ordering this thread's earlier memory operations before it (release,
// cluster scope).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];"
                 :: "r"(cluster_addr) : "memory");
}
// true once the phase of parity `parity` of this CTA's mbarrier has completed
// (acquire, cluster scope); never suspends the thread (the arrivals come from
// other CTAs, and a polling test reacts to them at once)
__device__ __forceinline__ bool mbar_test_wait(uint32_t addr, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(addr), "r"(parity) : "memory");
    return ok != 0;
}

// Barrier of the Q < 8 CTAs g0 .. g0 + Q - 1 of the cluster on the mbarrier
// `bar` (the same shared-memory offset in each of them, Q arrivals per
// phase).  Every thread of the CTA calls it.  The CTA barrier first orders the
// CTA's shared-memory accesses before thread 0's release arrivals; thread 0
// then waits (bounded) for the phase and the second CTA barrier passes its
// acquire on to every thread.
template <int Q>
__device__ __forceinline__ void group_sync(const uint32_t bar, const uint32_t g0,
                                           uint32_t& parity, const RaggedArgs& a) {
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int m = 0; m < Q; ++m) mbar_arrive_cluster(map_rank(bar, g0 + (uint32_t)m));
        bool ok = mbar_test_wait(bar, parity);
        for (int i = 0; i < a.wait_polls && !ok; ++i) {
            // after a timeout anywhere nothing waits any more
            if ((i & 1023) == 1023 && ld_status(a.status) != 0) break;
            ok = mbar_test_wait(bar, parity);
        }
        if (!ok && ld_status(a.status) == 0) atomicCAS(a.status, 0, SDFT_ERR_TIMEOUT);
    }
    parity ^= 1u;
    __syncthreads();
}

// pass 2's reads-done barrier for a group of Q < 8 CTAs: the arrivals are made
// once the remote values are in registers and used (after the step-0 register
// DFTs), then the wait, before Y is overwritten.
template <int Q>
struct GroupReadsDone {
    uint32_t bar, g0;
    uint32_t* parity;
    const RaggedArgs* a;
    __device__ __forceinline__ void after_gather() const {}
    __device__ __forceinline__ void before_scatter() const { group_sync<Q>(bar, g0, *parity, *a); }
};

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
        gyr[d + A * k2] = r;
        gyi[d + A * k2] = i;
    };
    pass2<CFG, ADJ>(st, smem, (uint32_t)__cvta_generic_to_shared(smem), tid, d, g0, tw, a.w, rd);
}

// Phase PHASE: the grid's groups of Q CTAs take the phase's transforms in
// turn (group g: items g, g + G, g + 2G, ..., G groups), all of equal size
// within a class, so no claims are needed; at the top of each item every CTA
// brings its share of the group's next transform into L2.
template <int Q, int PHASE, bool ADJ>
__device__ __forceinline__ void group_phase(const RaggedArgs& a, float* smem, const uint32_t rank,
                                            const uint32_t bar_a, const uint32_t bar_b) {
    static_assert(Q == (kRaggedCluster >> PHASE), "a phase's groups hold its routines' transforms");
    constexpr int PER = kRaggedCluster / Q;   // groups per cluster
    const uint32_t g0 = rank & ~(uint32_t)(Q - 1), q = rank & (uint32_t)(Q - 1);
    const int sub = (int)(rank / Q);
    const int stride = (int)(gridDim.x / kRaggedCluster) * PER;   // groups in the grid
    // coupled: the PER transforms a cluster runs at once share the hardware
    // cluster barrier (a group without a transform takes the barriers only);
    // otherwise every group synchronises alone with its mbarriers
    const bool coupled = Q == kRaggedCluster || ((a.coupled >> PHASE) & 1u);
    uint32_t pa = 0, pb = 0;
    auto sync_cluster = [] {
        cluster_arrive();
        cluster_wait();
    };
    auto sync_group = [&] { group_sync<Q>(bar_a, g0, pa, a); };
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
    while (coupled ? base < a.nitems[PHASE] : rec.x >= 0) {
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
        if (coupled) {
            const ClusterReadsDone rd{};
            switch (rec.x) {
                case kC16e: if constexpr (Q == 8) group_item<Cluster16e, ADJ>(a, rec, smem, q, g0, mid, sync_cluster, rd); break;
                case kC15q: if constexpr (Q == 8) group_item<Cluster15q, ADJ>(a, rec, smem, q, g0, mid, sync_cluster, rd); break;
                case kC15e: if constexpr (Q == 4) group_item<Cluster15e, ADJ>(a, rec, smem, q, g0, mid, sync_cluster, rd); break;
                case kC14q: if constexpr (Q == 4) group_item<Cluster14q, ADJ>(a, rec, smem, q, g0, mid, sync_cluster, rd); break;
                case kC14e: if constexpr (Q == 2) group_item<Cluster14e, ADJ>(a, rec, smem, q, g0, mid, sync_cluster, rd); break;
                case kC13: if constexpr (Q == 2) group_item<Cluster13, ADJ>(a, rec, smem, q, g0, mid, sync_cluster, rd); break;
                default:   // no transform for this group in this round
                    if (threadIdx.x == 0) tl->next[par] = nxt;
                    sync_cluster();
                    sync_cluster();
                    break;
            }
        } else if constexpr (Q < kRaggedCluster) {
            const GroupReadsDone<Q> rd{bar_b, g0, &pb, &a};
            switch (rec.x) {
                case kC15e: if constexpr (Q == 4) group_item<Cluster15e, ADJ>(a, rec, smem, q, g0, mid, sync_group, rd); break;
                case kC14q: if constexpr (Q == 4) group_item<Cluster14q, ADJ>(a, rec, smem, q, g0, mid, sync_group, rd); break;
                case kC14e: if constexpr (Q == 2) group_item<Cluster14e, ADJ>(a, rec, smem, q, g0, mid, sync_group, rd); break;
                case kC13: if constexpr (Q == 2) group_item<Cluster13, ADJ>(a, rec, smem, q, g0, mid, sync_group, rd); break;
                default: break;
            }
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
            case kR5D: row_tile<R5D, ADJ>(a, rec, smem); break;
            case kR6: row_tile<R6, ADJ>(a, rec, smem); break;
            case kR6D: row_tile<R6D, ADJ>(a, rec, smem); break;
            case kR7: row_tile<R7, ADJ>(a, rec, smem); break;
            case kR7D: row_tile<R7D, ADJ>(a, rec, smem); break;
            case kR8: row_tile<R8, ADJ>(a, rec, smem); break;
            case kR8D: row_tile<R8D, ADJ>(a, rec, smem); break;
            case kR8b: row_tile<R8b, ADJ>(a, rec, smem); break;
            case kR9: row_tile<R9, ADJ>(a, rec, smem); break;
            case kR9D: row_tile<R9D, ADJ>(a, rec, smem); break;
            case kR9b: row_tile<R9b, ADJ>(a, rec, smem); break;
            case kR10: row_tile<R10, ADJ>(a, rec, smem); break;
            case kR10D: row_tile<R10D, ADJ>(a, rec, smem); break;
            case kR11: row_tile<R11, ADJ>(a, rec, smem); break;
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
    RaggedTail* const tl = tail_of(smem);
    int4* const s_work = tl->work;
    uint64_t (&s_bar)[2][2] = tl->bar;
    const uint32_t rank = cluster_ctarank();
    const uint32_t b4a = (uint32_t)__cvta_generic_to_shared(&s_bar[0][0]);
    const uint32_t b4b = (uint32_t)__cvta_generic_to_shared(&s_bar[0][1]);
    const uint32_t b2a = (uint32_t)__cvta_generic_to_shared(&s_bar[1][0]);
    const uint32_t b2b = (uint32_t)__cvta_generic_to_shared(&s_bar[1][1]);
    if (threadIdx.x == 0) {
        mbar_init(b4a, 4);
        mbar_init(b4b, 4);
        mbar_init(b2a, 2);
        mbar_init(b2b, 2);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // every CTA of the cluster is running, with its barriers initialised,
    // before any of its shared memory is accessed from another CTA
    cluster_arrive();
    cluster_wait();
    if (a.nitems[0] > 0) group_phase<8, 0, ADJ>(a, smem, rank, 0u, 0u);
    if (a.nitems[1] > 0) group_phase<4, 1, ADJ>(a, smem, rank, b4a, b4b);
    if (a.nitems[2] > 0) group_phase<2, 2, ADJ>(a, smem, rank, b2a, b2b);
    if (a.nitems[3] > 0) row_phase<ADJ>(a, smem, s_work);
    // No CTA exits while another CTA of its cluster may still read its shared
    // memory or arrive on its mbarriers.  Group barriers guarantee that on the
    // normal path; after a wait has given up (SDFT_ERR_TIMEOUT) the CTAs of a
    // group no longer run in step, and this hardware barrier is what keeps
    // every CTA's shared memory alive until the whole cluster is done.
    cluster_arrive();
    cluster_wait();
}

}  // namespace rq
}  // namespace sdft
