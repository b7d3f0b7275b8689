// kernels_large.cu -- planar FP32 DFT for N = 32768 and 65536.
//
// A transform this long (256 or 512 KiB of FP32 pairs) exceeds one SM's
// registers and shared memory, so each CTA runs its transform as two passes
// over a CTA-private scratch slot (N = A * C, n = col + C * ntop,
// k = d + A * k2):
//   pass 1: for every column col < C, an A-point DFT over ntop, rotated by
//           W_N^{col * d}, written to scratch[d][col];
//   pass 2: for every row d < A, a C-point DFT over col of scratch[d][.],
//           written to y[d + A * k2].
// This is the same regrouping of the radix-2 factors of Eq. (6) that the
// row kernels use, with one extra level.  A persistent grid of one CTA per SM
// keeps the scratch slots (N * 8 bytes each) resident in L2, so the extra
// round trip mostly stays on chip.  Each transform is read completely (pass
// 1) before any of its output is written (pass 2), so in-place calls are safe.
//
// Inside each pass the sub-DFTs are run by the step engine with lanes mapped
// to columns (pass 1) or rows (pass 2), so every global access of a warp is
// a contiguous 128-byte line per plane.
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
    static constexpr int P1_FLOATS = 2 * A * TS1;
    static constexpr int STG = C + 1;                  // padded staging row
    static constexpr int P2_STAGE = 2 * TS2 * STG;
    static constexpr int P2_FLOATS = P2_STAGE + 2 * C * TS2;
    static constexpr size_t SMEM =
        (size_t)(P1_FLOATS > P2_FLOATS ? P1_FLOATS : P2_FLOATS) * sizeof(float);
    // twiddle tables: A-DFT step 0, C-DFT step 0, then W_N^{col * d}
    static constexpr int64_t TWA = 0, TWC = A, TWB = A + C, TW_TOTAL = A + C + (int64_t)N;
};

template <class CFG, bool ADJ>
__global__ void __launch_bounds__(CFG::THREADS, 1)
k_large(const float* xr, const float* xi, float* yr, float* yi, long long batch,
        const float2* __restrict__ tw, float2* scratch, const W64 w) {
    using SA = typename CFG::SA_;
    using SC = typename CFG::SC_;
    constexpr int A = CFG::A, C = CFG::C, N = CFG::N;
    extern __shared__ float4 smem4[];
    float* const sm = reinterpret_cast<float*>(smem4);
    const int lane = (int)threadIdx.x & 31;
    const int warp = (int)threadIdx.x >> 5;
    float* const scr_re = reinterpret_cast<float*>(scratch + (size_t)blockIdx.x * N);
    float* const scr_im = scr_re + N;

    auto sync = [] { __syncthreads(); };

    for (long long b = blockIdx.x; b < batch; b += gridDim.x) {
        const float* gxr = xr + b * (long long)N;
        const float* gxi = xi + b * (long long)N;
        float* gyr = yr + b * (long long)N;
        float* gyi = yi + b * (long long)N;

        // ---------------- pass 1: A-point DFTs down the columns ------------
        {
            const int ta = warp % SA::T;
            const int sub = (warp / SA::T) * 32 + lane;
            float* const x_re = sm;
            float* const x_im = sm + A * CFG::TS1;
            for (int tile = 0; tile < C / CFG::TS1; ++tile) {
                const int col = tile * CFG::TS1 + sub;
                auto ld = [&](int L, float& r, float& i) {
                    r = gxr[col + C * L];
                    i = gxi[col + C * L];
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
                sync();
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
}

template <int LOGA, int LOGC, class SA, class SC>
struct LargeCfgT : LargeCfg<LOGA, LOGC, SA, SC> {
    using SA_ = SA;
    using SC_ = SC;
};

template <class CFG>
cudaError_t large_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_large<CFG, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CFG::SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_large<CFG, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)CFG::SMEM);
}

template <class CFG>
int large_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_large<CFG, false>, CFG::THREADS,
                                                      CFG::SMEM) != cudaSuccess)
        return 0;
    return n;
}

template <class CFG>
cudaError_t large_launch(const LaunchArgs& a) {
    if (a.adj)
        return launch_kernel(k_large<CFG, true>, a.grid, CFG::THREADS, CFG::SMEM, a.stream, a.xr,
                             a.xi, a.yr, a.yi, a.batch, a.tw, a.scratch, a.w64);
    return launch_kernel(k_large<CFG, false>, a.grid, CFG::THREADS, CFG::SMEM, a.stream, a.xr,
                         a.xi, a.yr, a.yi, a.batch, a.tw, a.scratch, a.w64);
}

template <class CFG>
KernelInfo large_info(const char* name) {
    using SA = typename CFG::SA_;
    using SC = typename CFG::SC_;
    KernelInfo k = {};
    k.name = name;
    k.logn = CFG::LOGN;
    k.threads = CFG::THREADS;
    k.smem = CFG::SMEM;
    k.transforms_per_cta = 1;
    k.ntables = 3;
    k.tables[0] = TableDesc{CFG::A, (int64_t)1 << SA::lr(0), (int64_t)CFG::A >> SA::lr(0), CFG::TWA};
    k.tables[1] = TableDesc{CFG::C, (int64_t)1 << SC::lr(0), (int64_t)CFG::C >> SC::lr(0), CFG::TWC};
    k.tables[2] = TableDesc{CFG::N, CFG::A, CFG::C, CFG::TWB};
    k.tw_entries = CFG::TW_TOTAL;
    k.scratch_per_cta = CFG::N;
    k.launches = 1;
    k.prepare = large_prepare<CFG>;
    k.blocks_per_sm = large_blocks_per_sm<CFG>;
    k.launch = large_launch<CFG>;
    return k;
}

const KernelInfo* large_kernel(int logn) {
    using S256 = Steps<8, 4, 4, 4, 0>;   // 16 threads x 16 values, radix [16,16]
    using S128 = Steps<7, 4, 4, 3, 0>;   // 8 threads x 16 values, radix [16,8]
    static const KernelInfo k15 = large_info<LargeCfgT<8, 7, S256, S128>>(
        "N=32768: two passes per CTA through L2-resident scratch, 256 x 128, radix [16,16]x[16,8]");
    static const KernelInfo k16 = large_info<LargeCfgT<8, 8, S256, S256>>(
        "N=65536: two passes per CTA through L2-resident scratch, 256 x 256, radix [16,16]x[16,16]");
    switch (logn) {
        case 15: return &k15;
        case 16: return &k16;
        default: return nullptr;
    }
}

}  // namespace sdft
