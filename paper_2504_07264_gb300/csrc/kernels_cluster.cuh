// kernels_cluster.cuh -- one long transform (N = 16384 .. 65536) held in the
// distributed shared memory of Q CTAs of a thread-block cluster: the cluster
// primitives, the configurations and the two passes, shared by the uniform
// cluster kernel (cluster.cu) and the persistent work-queue kernel (ragged.cu).
//
// N = A * C, n = col + C * ntop, k = d + A * k2 (the regrouping of the radix-2
// factors of Eq. (6) used throughout the library):
//   pass 1: for every column col, the A-point DFT over ntop, rotated by
//           W_N^{col * d}                                 -> Y[d][col]
//   pass 2: for every row d, the C-point DFT over col     -> y[d + A * k2]
// CTA q of the Q runs pass 1 on columns [q C/Q, (q+1) C/Q) and keeps its part
// of Y in its own shared memory; after a cluster barrier it runs pass 2 on rows
// [q A/Q, (q+1) A/Q), reading each row's C values from the shared memory of
// all Q CTAs (ld.shared::cluster).  The intermediate never leaves the chip:
// HBM sees one read and one write of every point, as for short transforms.
// Each CTA holds N/Q = 8192 points, 256 threads x 32 values (or 4096 points,
// 128 threads x 32 values).
//
// Y is stored column-major, Y[c][d] at c * A + (d ^ (c mod 32)) (2c for
// 16-column tiles): in pass 1 a warp (32 columns, one d) writes 32 different
// banks, and in pass 2 a warp
// (32 consecutive rows d, one column) reads one whole 128-byte line of a
// remote CTA's shared memory per load.  Remote loads whose lanes touch
// different lines are split into one network transaction per line.
//
// Ordering: a second cluster barrier, split into arrive (after this CTA's
// remote reads) and wait (before this CTA overwrites Y), lets the pass-2 step-0
// register DFTs run while the barrier completes; when pass 2 returns, every
// remote read of this CTA's shared memory has finished.
#pragma once

#include "fft_core.cuh"

namespace sdft {

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_arrive() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// the address of the same shared-memory location in CTA `rank` of the cluster
// (a pure function of its operands: not volatile, so equal mappings are
// computed once)
__device__ __forceinline__ uint32_t map_rank(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
// Bring `bytes` (a multiple of 16, 16-byte aligned) of global memory into L2,
// asynchronously, with no destination in the SM.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ float ld_cluster(uint32_t addr) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}

template <int LOGA, int LOGC, int LOGQ, class SA, class SC, int THREADS_ = 256, int MINB_ = 0>
struct ClusterCfg {
    using SA_ = SA;
    using SC_ = SC;
    static constexpr int THREADS = THREADS_;
    // CTAs per SM: 64 K registers / (THREADS x 128) for 32 values per thread;
    // the 64-value forms give the count explicitly (3 x 128 threads, <= 170
    // registers each)
    static constexpr int MINB = MINB_ > 0 ? MINB_ : 512 / THREADS;
    static constexpr int Q = 1 << LOGQ;
    static constexpr int A = 1 << LOGA, C = 1 << LOGC, N = A * C, LOGN = LOGA + LOGC;
    static constexpr int LOGCQ = LOGC - LOGQ, CQ = 1 << LOGCQ;   // pass-1 columns per CTA
    static constexpr int AQ = A / Q;                              // pass-2 rows per CTA
    static_assert(SA::N == A && SC::N == C, "sub-DFT sizes");
    static_assert(SA::NS == 2 && SC::NS == 2, "two-step sub-DFTs");
    static_assert(CQ * SA::T == THREADS && AQ * SC::T == THREADS, "one CTA per column / row tile");
    static_assert(CQ >= 16 && AQ >= 32, "a warp covers 16 or 32 consecutive columns, 32 rows");
    static_assert(A % 32 == 0, "Y columns are whole 128-byte lines");
    // one buffer for the pass-1 exchange [L][CQ], Y and the pass-2 exchange
    // [L][AQ], each 2 * 8192 floats
    // Y swizzle: Y[c][d] at c * A + (d ^ swz(c)), swz(c) = c mod 32, or 2c
    // with 16-column tiles (a pass-1 warp then writes rows k and k + 1 of 16
    // columns: 2c keeps the 32 lanes on 32 banks)
    static constexpr int SWZ_SHIFT = CQ == 16 ? 1 : 0;
    __host__ __device__ static constexpr int swz(int c) { return (c << SWZ_SHIFT) & 31; }
    static constexpr int WORK_FLOATS = 2 * A * CQ;
    static_assert(2 * C * AQ == WORK_FLOATS, "the passes use equal buffers");
    static constexpr size_t SMEM = (size_t)WORK_FLOATS * sizeof(float);
    // The pass-1 rotation W_N^{col * k}, k = lo + P * d (P = the first A-step
    // radix, lo < P, d < R1 = the second), is taken as the product
    // W_N^{col * lo} * W_{N/P}^{col * d} of two small tables: a CTA's slices
    // of them (P + R1 rows of its CQ columns) stay in L1, where a full
    // [A][C] table would not.
    static constexpr int P = 1 << SA::lr(0), R1 = 1 << SA::lr(1);
    // twiddle tables: A-DFT step 0, C-DFT step 0, W_N^{col lo} at [lo][col],
    // W_{N/P}^{col d} at [d][col]
    static constexpr int64_t TWA = 0, TWC = A, TWB1 = A + C, TWB2 = TWB1 + (int64_t)P * C;
    static constexpr int64_t TW_TOTAL = TWB2 + (int64_t)R1 * C;
};

// Pass 1 from `ld` (step-0 source), Y into `work`.  Its first barrier orders
// the exchange writes after the previous transform's last reads of `work`.
// `mid` runs between the two steps (callers overlap other latency with it).
template <class CFG, bool ADJ, class LD, class MID>
__device__ __forceinline__ void pass1(LD ld, MID mid, float* const work, const int tid,
                                      const int col, const float2* __restrict__ tw, const W64& w) {
    using SA = typename CFG::SA_;
    constexpr int A = CFG::A, C = CFG::C, CQ = CFG::CQ;
    const int sub1 = tid % CQ, ta = tid / CQ;
    float* const x_re = work;                 // exchange [L][sub1]
    float* const x_im = work + A * CQ;
    float* const y_re = work;                 // Y[c][dd], swizzled
    float* const y_im = work + A * CQ;
    // With 16-column tiles a warp holds two rows L of the exchange; rows are
    // stored with bit 0 flipped when bit 5 is set, so that the step-0 writes
    // (rows d + 32 ta) and the step-1 reads (rows ta + 8 f + 32 i) of the two
    // half-warps fall on different banks.
    auto xrow = [](int L) { return CQ == 16 ? L ^ ((L >> 5) & 1) : L; };
    auto xw = [&](int L, float r, float i) {
        x_re[xrow(L) * CQ + sub1] = r;
        x_im[xrow(L) * CQ + sub1] = i;
    };
    auto xrd = [&](int L, float& r, float& i) {
        r = x_re[xrow(L) * CQ + sub1];
        i = x_im[xrow(L) * CQ + sub1];
    };
    auto twf = [&](int, int dd, int nl) -> float2 {
        return __ldg(tw + CFG::TWA + dd * (A >> SA::lr(0)) + nl);
    };
    auto none = [](int, float, float) {};
    float re[SA::E], im[SA::E];
    step_gather<SA, 0, ADJ>(re, im, ta, ld, xrd);
    __syncthreads();
    step_compute_scatter<SA, 0, ADJ>(re, im, ta, w, twf, xw, none);
    mid();
    __syncthreads();
    step_gather<SA, 1, ADJ>(re, im, ta, ld, xrd);
    __syncthreads();   // exchange reads done before Y (same memory) is written
    // last step: register DFTs, then output k = lo + P * d rotated by
    // W_N^{col k} = W_N^{col lo} * W_{N/P}^{col d} and written to Y
    using K = StepK<SA, 1>;
    static_assert(K::P == CFG::P && K::R == CFG::R1 && K::LAST, "two-step A-DFT");
    step_compute<SA, 1, ADJ>(re, im, w);
    float2 fac[K::R];
#pragma unroll
    for (int dd = 1; dd < K::R; ++dd) fac[dd] = __ldg(tw + CFG::TWB2 + dd * C + col);
#pragma unroll
    for (int f = 0; f < K::F; ++f) {
        const int lo = ta + SA::T * f;          // < P: the last step has no nl digit
        const float2 base = __ldg(tw + CFG::TWB1 + lo * C + col);
#pragma unroll
        for (int dd = 0; dd < K::R; ++dd) {
            const int reg = f * K::R + (SA::DIT ? dd : brevc(dd, K::LR));
            const int k = lo + K::P * dd;
            float2 wv = base;
            if (dd != 0) {
                wv.x = base.x * fac[dd].x - base.y * fac[dd].y;
                wv.y = base.x * fac[dd].y + base.y * fac[dd].x;
            }
            float r = re[reg], i = im[reg];
            rot<ADJ>(r, i, wv);
            y_re[sub1 * A + (k ^ CFG::swz(sub1))] = r;
            y_im[sub1 * A + (k ^ CFG::swz(sub1))] = i;
        }
    }
}

// The second barrier of pass 2 over the whole cluster: the arrive (release)
// follows this CTA's remote reads, the wait precedes the first write that
// reuses Y, and the step-0 register DFTs run in between.
struct ClusterReadsDone {
    __device__ __forceinline__ void after_gather() const { cluster_arrive(); }
    __device__ __forceinline__ void before_scatter() const { cluster_wait(); }
};

// Pass 2: rows of Y from every CTA of the cluster, results to `st`.  Every
// CTA's remote reads of this CTA's Y have finished when it returns.
// `rank0`: the cluster rank of the first of the Q CTAs that hold the transform.
// `rd`: the barrier that tells each CTA that the others' reads of its Y are
// done (after_gather() right after the remote loads, before_scatter() before
// Y is overwritten).
template <class CFG, bool ADJ, class ST, class RD = ClusterReadsDone>
__device__ __forceinline__ void pass2(ST st, float* const work, const uint32_t y_sh, const int tid,
                                      const int d, const uint32_t rank0,
                                      const float2* __restrict__ tw, const W64& w,
                                      const RD rd = RD{}) {
    using SC = typename CFG::SC_;
    constexpr int A = CFG::A, C = CFG::C, CQ = CFG::CQ, AQ = CFG::AQ;
    const int sub2 = tid % AQ, tc = tid / AQ;
    float* const x_re = work;                 // exchange [L][sub2]
    float* const x_im = work + C * AQ;
    // Column L of row d lives in CTA L / CQ at Y[L % CQ][d].  A step-0
    // element is L = c0 + C_s * i with c0 = tc + T * f < C_s <= CQ, so its
    // column is tc + ((L - tc) % CQ) and its CTA (L - tc) / CQ: L - tc is a
    // compile-time constant, and the address depends on the thread only
    // through tc and d (a few distinct bases, shared by many elements).
    static_assert((CFG::C >> SC::lr(0)) <= CQ, "a step-0 column stays within one CTA's columns");
    auto ld = [&](int L, float& r, float& i) {
        const int k = L - tc;
        const int c = tc + (k & (CQ - 1));
        const uint32_t a = map_rank(y_sh + 4u * (uint32_t)(c * A + (d ^ CFG::swz(c))),
                                    rank0 + (uint32_t)(k >> CFG::LOGCQ));
        r = ld_cluster(a);
        i = ld_cluster(a + 4u * (uint32_t)(A * CQ));
    };
    auto xw = [&](int L, float r, float i) {
        x_re[L * AQ + sub2] = r;
        x_im[L * AQ + sub2] = i;
    };
    auto xrd = [&](int L, float& r, float& i) {
        r = x_re[L * AQ + sub2];
        i = x_im[L * AQ + sub2];
    };
    auto twf = [&](int, int dd, int nl) -> float2 {
        return __ldg(tw + CFG::TWC + dd * (C >> SC::lr(0)) + nl);
    };
    float re[SC::E], im[SC::E];
    step_gather<SC, 0, ADJ>(re, im, tc, ld, xrd);
    rd.after_gather();     // this CTA's remote reads are done
    step_compute<SC, 0, ADJ>(re, im, w);
    rd.before_scatter();   // every CTA's reads of Y are done: Y may be overwritten
    step_scatter<SC, 0, ADJ>(re, im, tc, twf, xw, st);
    __syncthreads();
    step_gather<SC, 1, ADJ>(re, im, tc, ld, xrd);
    step_compute_scatter<SC, 1, ADJ>(re, im, tc, w, twf, xw, st);
}

using ClusterR256 = Steps<8, 5, 5, 3, 0>;   // 8 threads x 32 values, radix [32,8]
using ClusterR128 = Steps<7, 5, 5, 2, 0>;   // 4 threads x 32 values, radix [32,4]
using Cluster14 = ClusterCfg<7, 7, 1, ClusterR128, ClusterR128>;   // 128 x 128, Q = 2
using Cluster15 = ClusterCfg<8, 7, 2, ClusterR256, ClusterR128>;   // 256 x 128, Q = 4
using Cluster16 = ClusterCfg<8, 8, 3, ClusterR256, ClusterR256>;   // 256 x 256, Q = 8
// N = 32768 on clusters of 8 CTAs of 128 threads: 4096 points and 16 columns
// per CTA, four CTAs (of different transforms) per SM.  (The same form for
// N = 16384, clusters of 4, and N = 65536, clusters of 16, measured 241 and
// 158 Gpts/s against 234 and 176 for the 256-thread forms: at N = 65536 only
// 33 clusters of 16 fit and the pass-2 warps read 64-byte pieces.)
using Cluster15q = ClusterCfg<8, 7, 3, ClusterR256, ClusterR128, 128>;
// 64 values per thread: CTAs of 128 threads holding 8192 points, three per SM
// (24 K points in flight per SM instead of 16 K), the same A x C splits and
// Y layout as the 256-thread forms.
using ClusterE256 = Steps<8, 6, 5, 3, 0>;   // 4 threads x 64 values, radix [32,8]
using ClusterE128 = Steps<7, 6, 4, 3, 0>;   // 2 threads x 64 values, radix [16,8]
using Cluster16e = ClusterCfg<8, 8, 3, ClusterE256, ClusterE256, 128, 3>;   // 256 x 256, Q = 8
using Cluster15e = ClusterCfg<8, 7, 2, ClusterE256, ClusterE128, 128, 3>;   // 256 x 128, Q = 4
using Cluster14e = ClusterCfg<7, 7, 1, ClusterE128, ClusterE128, 128, 3>;   // 128 x 128, Q = 2
// 128-thread forms with 32 values per thread (4096 points per CTA), for the
// work-queue kernel: N = 16384 on four CTAs, N = 8192 on two
using ClusterR64 = Steps<6, 5, 3, 3, 0>;     // 2 threads x 32 values, radix [8,8]
using Cluster14q = ClusterCfg<7, 7, 2, ClusterR128, ClusterR128, 128>;   // 128 x 128, Q = 4
using Cluster13 = ClusterCfg<7, 6, 1, ClusterR128, ClusterR64, 128>;     // 128 x 64, Q = 2

}  // namespace sdft
