// kernels_large.cuh -- templates of the two-pass long-transform kernel
// (see kernels_large.cu for the method).
#pragma once

#include "fft_core.cuh"
#include "launch.h"

namespace sdft {

template <int LOGA, int LOGC, class SA, class SC>
struct LargeCfg {
    static constexpr int THREADS = 512, WARPS = 16;
    static constexpr int A = 1 << LOGA, C = 1 << LOGC, N = A * C, LOGN = LOGA + LOGC;
    static_assert(SA::N == A && SC::N == C, "sub-DFT sizes");
    static_assert(SA::NS == 2 && SC::NS == 2, "two-step sub-DFTs");
    static constexpr int TS1 = 32 * (WARPS / SA::T);   // columns per pass-1 tile
    static constexpr int TS2 = 32 * (WARPS / SC::T);   // rows per pass-2 tile
    static_assert(C % TS1 == 0 && A % TS2 == 0, "tiles");
    static constexpr int P1_TILE = 2 * A * TS1;             // one tile, both planes
    static constexpr int P1_FLOATS = 3 * P1_TILE;           // two prefetch buffers + exchange
    static constexpr int STG = C + 1;                  // padded staging row
    static constexpr int P2_STAGE = 2 * TS2 * STG;
    static constexpr int P2_FLOATS = P2_STAGE + 2 * C * TS2;
    static constexpr size_t SMEM =
        (size_t)(P1_FLOATS > P2_FLOATS ? P1_FLOATS : P2_FLOATS) * sizeof(float);
    // twiddle tables: A-DFT step 0, C-DFT step 0, then W_N^{col * d}
    static constexpr int64_t TWA = 0, TWC = A, TWB = A + C, TW_TOTAL = A + C + (int64_t)N;
};

// 16-byte asynchronous global -> shared copy (no register staging).
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int PENDING>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" :: "n"(PENDING) : "memory");
}

// One whole transform of CFG by the calling CTA (all CFG::THREADS threads):
// pass 1 into the CTA's scratch slot, pass 2 to the output.  `sm` is the
// CTA's dynamic shared memory (CFG::SMEM bytes).
template <class CFG, bool ADJ>
__device__ __forceinline__ void large_one(const float* gxr, const float* gxi, float* gyr,
                                          float* gyi, float* const scr_re, float* const scr_im,
                                          float* const sm, const float2* __restrict__ tw,
                                          const W64& w) {
    using SA = typename CFG::SA_;
    using SC = typename CFG::SC_;
    constexpr int A = CFG::A, C = CFG::C;
    const int lane = (int)threadIdx.x & 31;
    const int warp = (int)threadIdx.x >> 5;
    auto sync = [] { __syncthreads(); };
    // ---------------- pass 1: A-point DFTs down the columns ------------
    // Column tiles (A rows x TS1 columns, both planes) are copied into one
    // of two shared buffers with cp.async while the previous tile is being
    // transformed, so the HBM reads overlap the register DFTs.
    {
        const int ta = warp % SA::T;
        const int sub = (warp / SA::T) * 32 + lane;
        constexpr int TILES = C / CFG::TS1;
        constexpr int CHUNKS = A * CFG::TS1 / 4;         // 16-byte chunks per plane
        float* const x_re = sm + 2 * CFG::P1_TILE;       // exchange
        float* const x_im = x_re + A * CFG::TS1;
        auto issue = [&](int tile) {
            float* const buf = sm + (tile & 1) * CFG::P1_TILE;
            const int col0 = tile * CFG::TS1;
            for (int u = (int)threadIdx.x; u < CHUNKS; u += CFG::THREADS) {
                const int L = u / (CFG::TS1 / 4), q = u % (CFG::TS1 / 4);
                cp_async16(buf + L * CFG::TS1 + 4 * q, gxr + col0 + 4 * q + (long long)C * L);
                cp_async16(buf + A * CFG::TS1 + L * CFG::TS1 + 4 * q,
                           gxi + col0 + 4 * q + (long long)C * L);
            }
            cp_async_commit();
        };
        issue(0);
        for (int tile = 0; tile < TILES; ++tile) {
            if (tile + 1 < TILES) {
                issue(tile + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            sync();                                      // this tile's copies visible
            const float* const b_re = sm + (tile & 1) * CFG::P1_TILE;
            const float* const b_im = b_re + A * CFG::TS1;
            const int col = tile * CFG::TS1 + sub;
            auto ld = [&](int L, float& r, float& i) {
                r = b_re[L * CFG::TS1 + sub];
                i = b_im[L * CFG::TS1 + sub];
            };
            auto xw = [&](int L, float r, float i) {
                x_re[L * CFG::TS1 + sub] = r;
                x_im[L * CFG::TS1 + sub] = i;
            };
            auto xrd = [&](int L, float& r, float& i) {
                r = x_re[L * CFG::TS1 + sub];
                i = x_im[L * CFG::TS1 + sub];
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
            sync();                                      // buffer and exchange free again
        }
    }
    // scratch writes of pass 1 visible to the whole CTA (the last sync above)

    // ---------------- pass 2: C-point DFTs along the rows --------------
    {
        const int tc = warp % SC::T;
        const int sub = (warp / SC::T) * 32 + lane;
        float* const g_re = sm;                                  // staged rows
        float* const g_im = sm + CFG::TS2 * CFG::STG;
        float* const x_re = sm + CFG::P2_STAGE;                  // exchange
        float* const x_im = x_re + C * CFG::TS2;
        for (int tile = 0; tile < A / CFG::TS2; ++tile) {
            // stage TS2 contiguous scratch rows into padded shared memory
            const float4* src_re = reinterpret_cast<const float4*>(scr_re + tile * CFG::TS2 * C);
            const float4* src_im = reinterpret_cast<const float4*>(scr_im + tile * CFG::TS2 * C);
            for (int u = (int)threadIdx.x; u < CFG::TS2 * C / 4; u += CFG::THREADS) {
                const float4 a = src_re[u];
                const float4 c = src_im[u];
                const int row = (4 * u) / C, cc = (4 * u) % C;
                float* dr = g_re + row * CFG::STG + cc;
                float* di = g_im + row * CFG::STG + cc;
                dr[0] = a.x; dr[1] = a.y; dr[2] = a.z; dr[3] = a.w;
                di[0] = c.x; di[1] = c.y; di[2] = c.z; di[3] = c.w;
            }
            sync();
            const int d = tile * CFG::TS2 + sub;
            auto ld = [&](int L, float& r, float& i) {
                r = g_re[sub * CFG::STG + L];
                i = g_im[sub * CFG::STG + L];
            };
            auto xw = [&](int L, float r, float i) {
                x_re[L * CFG::TS2 + sub] = r;
                x_im[L * CFG::TS2 + sub] = i;
            };
            auto xrd = [&](int L, float& r, float& i) {
                r = x_re[L * CFG::TS2 + sub];
                i = x_im[L * CFG::TS2 + sub];
            };
            auto twf = [&](int, int dd, int nl) -> float2 {
                return __ldg(tw + CFG::TWC + dd * (C >> SC::lr(0)) + nl);
            };
            auto st = [&](int k2, float r, float i) {
                gyr[d + A * k2] = r;
                gyi[d + A * k2] = i;
            };
            run_steps<SC, ADJ>(tc, w, ld, xw, xrd, twf, st, sync);
            sync();
        }
    }
}

template <class CFG, bool ADJ>
__global__ void __launch_bounds__(CFG::THREADS, 1)
k_large(const float* xr, const float* xi, float* yr, float* yi, long long batch,
        const float2* __restrict__ tw, float2* scratch, const W64 w) {
    constexpr int N = CFG::N;
    extern __shared__ float4 smem4[];
    float* const sm = reinterpret_cast<float*>(smem4);
    float* const scr_re = reinterpret_cast<float*>(scratch + (size_t)blockIdx.x * N);
    float* const scr_im = scr_re + N;
    for (long long b = blockIdx.x; b < batch; b += gridDim.x) {
        const long long row = b * (long long)N;
        large_one<CFG, ADJ>(xr + row, xi + row, yr + row, yi + row, scr_re, scr_im, sm, tw, w);
    }
}

template <int LOGA, int LOGC, class SA, class SC>
struct LargeCfgT : LargeCfg<LOGA, LOGC, SA, SC> {
    using SA_ = SA;
    using SC_ = SC;
};


}  // namespace sdft
