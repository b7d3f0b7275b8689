// kernels_items.cuh -- long transforms (N = 16384 .. 65536) as independent
// work items of a persistent kernel.
//
// N = A * C, n = col + C * ntop, k = d + A * k2 (the regrouping of the radix-2
// factors of Eq. (6) used throughout the library):
//   pass-1 item (transform t, column tile j): the A-point DFTs over ntop of
//     columns [32j, 32j+32), each rotated by W_N^{col * d}, written to the
//     transform's scratch slot as scratch[d][col];
//   pass-2 item (transform t, row tile j): once every pass-1 item of t has
//     finished, the C-point DFTs over col of rows [32j, 32j+32) of the slot,
//     written to y[d + A * k2].
// Items of different transforms, and the two passes of one transform, run on
// different CTAs at the same time, so loads, arithmetic and stores of many
// transforms overlap across the GPU.  Each item is one 256-thread CTA tile:
// 8 threads per sub-DFT (the warp index), lanes = the 32 columns (pass 1) or
// rows (pass 2), so every global access of a warp is one 128-byte line per
// plane.  Scratch is read with L1-bypassing loads because other SMs wrote it.
#pragma once

#include "fft_core.cuh"
#include "launch.h"

namespace sdft {

template <int LOGA, int LOGC, class SA, class SC>
struct ItemCfg {
    using SA_ = SA;
    using SC_ = SC;
    static constexpr int THREADS = 256, WARPS = 8;
    static constexpr int A = 1 << LOGA, C = 1 << LOGC, N = A * C, LOGN = LOGA + LOGC;
    static_assert(SA::N == A && SC::N == C, "sub-DFT sizes");
    static_assert(SA::T == WARPS && SC::T == WARPS, "one warp per sub-DFT thread index");
    static_assert(SA::NS == 2 && SC::NS == 2, "two-step sub-DFTs");
    static constexpr int TS = 32;                   // columns / rows per tile (lanes)
    static constexpr int TILES1 = C / TS, TILES2 = A / TS;
    static constexpr int STG = C + 1;               // padded staging row (pass 2)
    static constexpr int P1_FLOATS = 2 * A * TS;    // exchange
    static constexpr int P2_FLOATS = 2 * TS * STG;  // staging, then exchange (aliased)
    static_assert(2 * C * TS <= P2_FLOATS, "pass-2 exchange fits the staging area");
    static constexpr size_t SMEM =
        (size_t)(P1_FLOATS > P2_FLOATS ? P1_FLOATS : P2_FLOATS) * sizeof(float);
    // twiddle tables: A-DFT step 0, C-DFT step 0, then W_N^{col * d} at [d][col]
    static constexpr int64_t TWA = 0, TWC = A, TWB = A + C, TW_TOTAL = A + C + (int64_t)N;
};

// pass-1 item: column tile `tile` of the transform at gxr/gxi into its slot.
template <class CFG, bool ADJ>
__device__ __forceinline__ void item_pass1(const float* gxr, const float* gxi, float* scr_re,
                                           float* scr_im, const int tile, float* const sm,
                                           const float2* __restrict__ tw, const W64& w) {
    using SA = typename CFG::SA_;
    constexpr int A = CFG::A, C = CFG::C, TS = CFG::TS;
    const int sub = (int)threadIdx.x & 31;
    const int ta = (int)threadIdx.x >> 5;
    const int col = tile * TS + sub;
    float* const x_re = sm;
    float* const x_im = sm + A * TS;
    auto sync = [] { __syncthreads(); };
    auto ld = [&](int L, float& r, float& i) {
        r = gxr[col + C * L];
        i = gxi[col + C * L];
    };
    auto xw = [&](int L, float r, float i) {
        x_re[L * TS + sub] = r;
        x_im[L * TS + sub] = i;
    };
    auto xrd = [&](int L, float& r, float& i) {
        r = x_re[L * TS + sub];
        i = x_im[L * TS + sub];
    };
    auto twf = [&](int, int d, int nl) -> float2 {
        return __ldg(tw + CFG::TWA + d * (A >> SA::lr(0)) + nl);
    };
    auto st = [&](int k, float r, float i) {
        rot<ADJ>(r, i, __ldg(tw + CFG::TWB + (int64_t)k * C + col));
        scr_re[k * C + col] = r;
        scr_im[k * C + col] = i;
    };
    run_steps<SA, ADJ>(ta, w, ld, xw, xrd, twf, st, sync);
}

// pass-2 item: row tile `tile` of the slot into the output at gyr/gyi.
template <class CFG, bool ADJ>
__device__ __forceinline__ void item_pass2(const float* scr_re, const float* scr_im, float* gyr,
                                           float* gyi, const int tile, float* const sm,
                                           const float2* __restrict__ tw, const W64& w) {
    using SC = typename CFG::SC_;
    constexpr int A = CFG::A, C = CFG::C, TS = CFG::TS, STG = CFG::STG;
    const int sub = (int)threadIdx.x & 31;
    const int tc = (int)threadIdx.x >> 5;
    float* const g_re = sm;
    float* const g_im = sm + TS * STG;
    float* const x_re = sm;                  // exchange reuses the staging area
    float* const x_im = sm + C * TS;
    auto sync = [] { __syncthreads(); };
    // stage TS contiguous slot rows (written by other SMs: bypass L1); one
    // float per lane so that consecutive lanes write consecutive banks
    const float* src_re = scr_re + tile * TS * C;
    const float* src_im = scr_im + tile * TS * C;
#pragma unroll 8
    for (int u = (int)threadIdx.x; u < TS * C; u += CFG::THREADS) {
        const int row = u / C, cc = u % C;
        g_re[row * STG + cc] = __ldcg(src_re + u);
        g_im[row * STG + cc] = __ldcg(src_im + u);
    }
    sync();
    const int d = tile * TS + sub;
    auto ld = [&](int L, float& r, float& i) {
        r = g_re[sub * STG + L];
        i = g_im[sub * STG + L];
    };
    auto xw = [&](int L, float r, float i) {
        x_re[L * TS + sub] = r;
        x_im[L * TS + sub] = i;
    };
    auto xrd = [&](int L, float& r, float& i) {
        r = x_re[L * TS + sub];
        i = x_im[L * TS + sub];
    };
    auto twf = [&](int, int dd, int nl) -> float2 {
        return __ldg(tw + CFG::TWC + dd * (C >> SC::lr(0)) + nl);
    };
    auto st = [&](int k2, float r, float i) {
        gyr[d + A * k2] = r;
        gyi[d + A * k2] = i;
    };
    run_steps<SC, ADJ, true>(tc, w, ld, xw, xrd, twf, st, sync);
}

}  // namespace sdft
