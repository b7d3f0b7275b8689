// kernels_rows.cuh -- batched planar FP32 DFT, one transform per thread group.
//
// Each transform (a contiguous row of N floats in each of xr, xi) is owned by
// T = N / E threads of one CTA; a CTA holds G transforms.  Step 0 reads the
// row straight from global memory with the thread <-> element map of the
// step engine (consecutive threads read consecutive elements, so every warp
// access is a full, aligned 128-byte line per plane); later steps exchange
// through padded shared memory; the last step writes natural order straight
// to global memory.  For N <= 32 one thread owns a whole row and moves it
// with 16-byte vector loads and stores.
//
// The kernel is templated on direction: the forward kernel applies the
// rotations W of Eq. (1); the adjoint kernel (E_2N^T) applies their
// conjugates, i.e. the transposed 2x2 blocks omega^(i,q)^T.
#pragma once

#include "../../include/sdft.h"
#include "fft_core.cuh"
#include "launch.h"

namespace sdft {

template <int LOGN, int LOGE, int LR0, int LR1, int LR2, int G_, int SBX_ = 0, int MINB_ = 1,
          bool DIT = false, bool SWZ_ = false>
struct RowCfg {
    using S = Steps<LOGN, LOGE, LR0, LR1, LR2, DIT>;
    static constexpr int G = G_;
    static constexpr int THREADS = S::T * G;
    static constexpr int MINB = MINB_;
    // SWZ: the exchange is XOR-swizzled (swz32) rather than padded (pad32),
    // so it takes exactly N words per plane (conflict-free for the splits it
    // is used with: every step's columns 32 lanes apart or consecutive)
    static constexpr bool SWZ = SWZ_;
    static constexpr int PLANE = S::N + (SWZ ? 0 : (S::N >> 5));
    static constexpr int BUF = 2 * PLANE + SBX_;
    static constexpr size_t SMEM = S::NS > 1 ? (size_t)G * BUF * sizeof(float) : 0;
    // Step-0 rotations W_N^{nl d} (d < R0, nl < Q0 = N / R0).  For Q0 >= 64
    // (N >= 2048) the full table (N entries, 16 .. 128 KiB) does not stay in
    // L1 beside 66 KiB of shared memory per CTA, so it is factored,
    // d = dl + 8 dh: W_N^{nl dl} ([dl][nl], dl < 8) times W_{N/8}^{nl dh}
    // ([dh][nl], dh < R0 / 8), one extra complex product per rotation.
    static constexpr int R0 = 1 << S::lr(0), Q0 = S::N / R0;
    static constexpr bool FACT = S::NS > 1 && R0 >= 16 && Q0 >= 64;
    static constexpr int64_t TW0 = 0;
    static constexpr int64_t TWB = 8 * (int64_t)Q0;          // [dh][nl] when FACT
    static constexpr int64_t TW1 =
        S::NS > 1 ? (FACT ? TWB + (R0 / 8) * (int64_t)Q0 : S::tw_entries(0)) : 0;
    static constexpr int64_t TW_TOTAL = TW1 + (S::NS > 2 ? S::tw_entries(1) : 0);
    static_assert(THREADS <= 1024, "CTA too large");
    static_assert(S::T <= 32 || G == 1 || THREADS <= 1024, "");
};

// The rotation of step s for output digit d of column group nl (see RowCfg).
template <class CFG>
__device__ __forceinline__ float2 rows_twiddle(const float2* __restrict__ tw, const int s,
                                               const int d, const int nl) {
    using S = typename CFG::S;
    if constexpr (CFG::FACT) {
        if (s == 0) {
            const int dl = d & 7, dh = d >> 3;
            if (dh == 0) return __ldg(tw + CFG::TW0 + dl * CFG::Q0 + nl);
            const float2 b = __ldg(tw + CFG::TWB + dh * CFG::Q0 + nl);
            if (dl == 0) return b;
            const float2 a = __ldg(tw + CFG::TW0 + dl * CFG::Q0 + nl);
            return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
        }
    }
    const int64_t off = (s == 0) ? CFG::TW0 : CFG::TW1;
    const int q = (s == 0) ? (S::N >> S::lr(0)) : (S::N >> (S::lr(0) + S::lr(1)));
    return __ldg(tw + off + (int64_t)d * q + nl);
}

// The tables rows_twiddle reads, for plan creation; returns their count.
template <class CFG>
int rows_tables(TableDesc* t) {
    using S = typename CFG::S;
    int n = 0;
    if (S::NS > 1) {
        const int64_t nn = S::N;
        if (CFG::FACT) {
            t[n++] = TableDesc{nn, 8, CFG::Q0, CFG::TW0};
            t[n++] = TableDesc{nn / 8, CFG::R0 / 8, CFG::Q0, CFG::TWB};
        } else {
            t[n++] = TableDesc{nn, (int64_t)1 << S::lr(0), nn >> S::lr(0), CFG::TW0};
        }
        if (S::NS > 2) {
            const int64_t m1 = nn >> S::lr(0);
            t[n++] = TableDesc{m1, (int64_t)1 << S::lr(1), m1 >> S::lr(1), CFG::TW1};
        }
    }
    return n;
}

// One tile of CFG: group g (the caller's `t`, `s_re`, `s_im` belong to it)
// transforms the row at gxr/gxi into gyr/gyi when `active`.  Every thread of
// the CTA must call this (inactive groups still take part in the barriers).
template <class CFG, bool ADJ>
__device__ __forceinline__ void rows_tile(const float* gxr, const float* gxi, float* gyr,
                                          float* gyi, const bool active, const int t,
                                          float* const s_re, float* const s_im,
                                          const float2* __restrict__ tw, const W64& w) {
    using S = typename CFG::S;
    auto sync = [] {
        if constexpr (S::T <= 32) __syncwarp();
        else __syncthreads();
    };
    auto xw = [&](int L, float r, float i) {
        const int p = CFG::SWZ ? swz32(L) : pad32(L);
        s_re[p] = r;
        s_im[p] = i;
    };
    auto xrd = [&](int L, float& r, float& i) {
        const int p = CFG::SWZ ? swz32(L) : pad32(L);
        r = s_re[p];
        i = s_im[p];
    };
    auto twf = [&](int s, int d, int nl) -> float2 { return rows_twiddle<CFG>(tw, s, d, nl); };
    if constexpr (S::T == 1) {
        // whole row per thread: vector loads into registers, then the step
        // engine reads them by compile-time index.
        constexpr int N = S::N;
        float ar[N], ai[N];
        if (active) {
            if constexpr (N >= 4) {
#pragma unroll
                for (int v = 0; v < N / 4; ++v) {
                    const float4 a = reinterpret_cast<const float4*>(gxr)[v];
                    const float4 c = reinterpret_cast<const float4*>(gxi)[v];
                    ar[4 * v] = a.x; ar[4 * v + 1] = a.y; ar[4 * v + 2] = a.z; ar[4 * v + 3] = a.w;
                    ai[4 * v] = c.x; ai[4 * v + 1] = c.y; ai[4 * v + 2] = c.z; ai[4 * v + 3] = c.w;
                }
            } else {
                const float2 a = reinterpret_cast<const float2*>(gxr)[0];
                const float2 c = reinterpret_cast<const float2*>(gxi)[0];
                ar[0] = a.x; ar[1] = a.y;
                ai[0] = c.x; ai[1] = c.y;
            }
        } else {
#pragma unroll
            for (int v = 0; v < N; ++v) { ar[v] = 0.f; ai[v] = 0.f; }
        }
        float orr[N], oi[N];
        auto ld = [&](int L, float& r, float& i) { r = ar[L]; i = ai[L]; };
        auto st = [&](int k, float r, float i) { orr[k] = r; oi[k] = i; };
        run_steps<S, ADJ>(t, w, ld, xw, xrd, twf, st, sync);
        if (active) {
            if constexpr (N >= 4) {
#pragma unroll
                for (int v = 0; v < N / 4; ++v) {
                    reinterpret_cast<float4*>(gyr)[v] =
                        make_float4(orr[4 * v], orr[4 * v + 1], orr[4 * v + 2], orr[4 * v + 3]);
                    reinterpret_cast<float4*>(gyi)[v] =
                        make_float4(oi[4 * v], oi[4 * v + 1], oi[4 * v + 2], oi[4 * v + 3]);
                }
            } else {
                reinterpret_cast<float2*>(gyr)[0] = make_float2(orr[0], orr[1]);
                reinterpret_cast<float2*>(gyi)[0] = make_float2(oi[0], oi[1]);
            }
        }
    } else {
        auto ld = [&](int L, float& r, float& i) {
            if (active) { r = gxr[L]; i = gxi[L]; }
            else { r = 0.f; i = 0.f; }
        };
        auto st = [&](int k, float r, float i) {
            if (active) { gyr[k] = r; gyi[k] = i; }
        };
        run_steps<S, ADJ>(t, w, ld, xw, xrd, twf, st, sync);
        if constexpr (S::NS > 1) sync();  // last reads done before the next tile writes
    }
}

template <class CFG, bool ADJ>
__global__ void __launch_bounds__(CFG::THREADS, CFG::MINB)
k_rows(const float* xr, const float* xi, float* yr, float* yi, long long batch,
       const float2* __restrict__ tw, const W64 w) {
    using S = typename CFG::S;
    extern __shared__ float4 smem4[];
    float* const smem = reinterpret_cast<float*>(smem4);
    const int t = (int)threadIdx.x & (S::T - 1);
    const int g = (int)threadIdx.x >> S::LOGT;
    float* const s_re = smem + g * CFG::BUF;
    float* const s_im = s_re + CFG::PLANE;
    const long long ntiles = (batch + CFG::G - 1) / CFG::G;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long b = tile * CFG::G + g;
        const bool active = b < batch;
        const long long row = (active ? b : 0) * (long long)S::N;
        rows_tile<CFG, ADJ>(xr + row, xi + row, yr + row, yi + row, active, t, s_re, s_im, tw, w);
    }
}

template <class CFG>
cudaError_t rows_prepare() {
    cudaError_t e = cudaSuccess;
    if (CFG::SMEM > 48 * 1024) {
        e = cudaFuncSetAttribute(k_rows<CFG, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)CFG::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_rows<CFG, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)CFG::SMEM);
    }
    return e;
}

template <class CFG>
int rows_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rows<CFG, false>, CFG::THREADS,
                                                      CFG::SMEM) != cudaSuccess)
        return 0;
    return n;
}

template <class CFG>
cudaError_t rows_launch(const LaunchArgs& a) {
    if (a.adj)
        return launch_kernel(k_rows<CFG, true>, a.grid, CFG::THREADS, CFG::SMEM, a.stream, a.xr,
                             a.xi, a.yr, a.yi, a.batch, a.tw, a.w64);
    return launch_kernel(k_rows<CFG, false>, a.grid, CFG::THREADS, CFG::SMEM, a.stream, a.xr,
                         a.xi, a.yr, a.yi, a.batch, a.tw, a.w64);
}

// Name, shape and twiddle tables of a row configuration (no launch hooks).
template <class CFG>
KernelInfo rows_shape(const char* name) {
    using S = typename CFG::S;
    KernelInfo k = {};
    k.name = name;
    k.logn = S::LOGN;
    k.threads = CFG::THREADS;
    k.smem = CFG::SMEM;
    k.transforms_per_cta = CFG::G;
    k.ntables = rows_tables<CFG>(k.tables);
    k.tw_entries = CFG::TW_TOTAL;
    k.scratch_per_cta = 0;
    k.launches = 1;
    return k;
}

template <class CFG>
KernelInfo rows_info(const char* name) {
    KernelInfo k = rows_shape<CFG>(name);
    k.prepare = rows_prepare<CFG>;
    k.blocks_per_sm = rows_blocks_per_sm<CFG>;
    k.launch = rows_launch<CFG>;
    return k;
}

// ---------------------------------------------------------------------------
// Prefetching variant: a CTA of 128 threads holds G transforms (4096 points)
// per tile, and the next tile's rows arrive by 1-D bulk copies (TMA) into a
// shared input buffer while the current tile runs its register steps, so
// HBM reads overlap computation inside one CTA as well as across the three
// CTAs of an SM.  Step 0 gathers from that buffer; the other steps are those
// of k_rows; the last step stores straight to global memory.
// ---------------------------------------------------------------------------
template <class RC, int MINB_ = 3, int PART_ = 1>
struct RowPfCfg {
    using RC_ = RC;
    using S = typename RC::S;
    static constexpr int G = RC::G;
    static constexpr int THREADS = RC::THREADS;
    static constexpr int MINB = MINB_;
    static constexpr int N = S::N;
    // PART > 1 (one transform per tile): only the first N / PART points of the
    // next row are prefetched, the rest are loaded when the tile starts, so
    // that the input buffer leaves room for a second CTA (N = 8192) or fits
    // beside the exchange buffer at all (N = 16384).
    static constexpr int PART = PART_;
    static constexpr int PN = N / PART;
    static_assert(PART == 1 || G == 1, "partial prefetch for one transform per tile");
    static constexpr int IN_FLOATS = 2 * G * PN;          // [re: G x PN][im: G x PN]
    static constexpr size_t SMEM = (size_t)(IN_FLOATS + G * RC::BUF) * sizeof(float);
    static_assert(S::NS > 1, "transforms with a shared-memory exchange");
    static_assert((N * 4) % 16 == 0, "bulk copies of whole rows");
};

template <class CFG, bool ADJ>
__global__ void __launch_bounds__(CFG::THREADS, CFG::MINB)
k_rows_pf(const float* xr, const float* xi, float* yr, float* yi, long long batch,
          const float2* __restrict__ tw, const W64 w, int* status) {
    using RC = typename CFG::RC_;
    using S = typename CFG::S;
    constexpr int N = CFG::N, G = CFG::G;
    extern __shared__ float4 smem4[];
    float* const in_re = reinterpret_cast<float*>(smem4);
    float* const in_im = in_re + G * CFG::PN;
    __shared__ __align__(8) uint64_t mbar;
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
    const int tid = (int)threadIdx.x;
    const int t = tid & (S::T - 1);
    const int g = tid >> S::LOGT;
    float* const s_re = in_re + CFG::IN_FLOATS + g * RC::BUF;
    float* const s_im = s_re + RC::PLANE;
    const long long ntiles = (batch + G - 1) / G;
    // thread 0: the rows of tile `k` into the input buffer
    auto load = [&](long long k) {
        const long long first = k * G;
        const int cnt = (int)((batch - first < G) ? (batch - first) : G);
        const uint32_t bytes = (uint32_t)cnt * CFG::PN * 4u;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(mb), "r"(2u * bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"((uint32_t)__cvta_generic_to_shared(in_re)), "l"(xr + first * N), "r"(bytes),
                        "r"(mb) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"((uint32_t)__cvta_generic_to_shared(in_im)), "l"(xi + first * N), "r"(bytes),
                        "r"(mb) : "memory");
        if constexpr (CFG::PART > 1) {
            // the rest of the row, loaded from global memory when the tile
            // starts, into L2 meanwhile
            constexpr uint32_t rest = (uint32_t)(N - CFG::PN) * 4u;
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                         :: "l"(xr + first * N + CFG::PN), "r"(rest) : "memory");
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                         :: "l"(xi + first * N + CFG::PN), "r"(rest) : "memory");
        }
    };
    // bounded wait for the phase of parity `ph`
    auto wait = [&](uint32_t ph) {
        for (int i = 0; i < (1 << 21); ++i) {
            uint32_t ok;
            asm volatile("{\n\t.reg .pred p;\n\t"
                         "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                         "selp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(ok) : "r"(mb), "r"(ph) : "memory");
            if (ok) return true;
        }
        return false;
    };
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(mb) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    bool pending = false;   // thread 0: a tile load not yet waited for
    if (tid == 0 && blockIdx.x < ntiles) { load(blockIdx.x); pending = true; }
    uint32_t ph = 0;
    auto xw = [&](int L, float r, float i) {
        const int p = RC::SWZ ? swz32(L) : pad32(L);
        s_re[p] = r;
        s_im[p] = i;
    };
    auto xrd = [&](int L, float& r, float& i) {
        const int p = RC::SWZ ? swz32(L) : pad32(L);
        r = s_re[p];
        i = s_im[p];
    };
    auto twf = [&](int s, int d, int nl) -> float2 { return rows_twiddle<RC>(tw, s, d, nl); };
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        if (__syncthreads_or(!wait(ph))) {      // gave up: record it and stop
            if (tid == 0) atomicCAS(status, 0, SDFT_ERR_TIMEOUT);
            break;
        }
        ph ^= 1;
        if (tid == 0) pending = false;
        const long long b = tile * G + g;
        const bool active = b < batch;
        float* const gyr = yr + (active ? b : 0) * (long long)N;
        float* const gyi = yi + (active ? b : 0) * (long long)N;
        const float* const gxr = xr + (active ? b : 0) * (long long)N;
        const float* const gxi = xi + (active ? b : 0) * (long long)N;
        auto ld = [&](int L, float& r, float& i) {
            if (CFG::PART == 1 || L < CFG::PN) {
                r = in_re[g * CFG::PN + L];
                i = in_im[g * CFG::PN + L];
            } else {
                r = gxr[L];
                i = gxi[L];
            }
        };
        auto st = [&](int k, float r, float i) {
            if (active) { gyr[k] = r; gyi[k] = i; }
        };
        // the first barrier (after the step-0 gather) frees the input buffer
        // for the next tile and orders this tile's exchange writes after the
        // previous tile's last exchange reads
        int nsync = 0;
        const long long next = tile + gridDim.x;
        auto sync = [&] {
            __syncthreads();
            if (nsync++ == 0 && tid == 0 && next < ntiles) { load(next); pending = true; }
        };
        run_steps<S, ADJ, true>(t, w, ld, xw, xrd, twf, st, sync);
    }
    if (tid == 0 && pending) wait(ph);   // no tile load left in flight (bounded)
}

template <class CFG>
cudaError_t rows_pf_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_rows_pf<CFG, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CFG::SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_rows_pf<CFG, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)CFG::SMEM);
}

template <class CFG>
int rows_pf_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rows_pf<CFG, false>, CFG::THREADS,
                                                      CFG::SMEM) != cudaSuccess)
        return 0;
    return n;
}

template <class CFG>
cudaError_t rows_pf_launch(const LaunchArgs& a) {
    if (a.adj)
        return launch_kernel(k_rows_pf<CFG, true>, a.grid, CFG::THREADS, CFG::SMEM, a.stream, a.xr,
                             a.xi, a.yr, a.yi, a.batch, a.tw, a.w64, a.status);
    return launch_kernel(k_rows_pf<CFG, false>, a.grid, CFG::THREADS, CFG::SMEM, a.stream, a.xr,
                         a.xi, a.yr, a.yi, a.batch, a.tw, a.w64, a.status);
}

template <class CFG>
KernelInfo rows_pf_info(const char* name) {
    KernelInfo k = rows_shape<typename CFG::RC_>(name);
    k.smem = CFG::SMEM;
    k.prepare = rows_pf_prepare<CFG>;
    k.blocks_per_sm = rows_pf_blocks_per_sm<CFG>;
    k.launch = rows_pf_launch<CFG>;
    return k;
}

// ---------------------------------------------------------------------------
// Transposing variant for one thread per transform (N = 16, 32).  With each
// lane loading its own row, a warp's 16-byte loads touch 32 different lines
// (lanes N * 4 bytes apart), and the L1 serves one line per cycle.  Here each
// warp moves the rows of its 32 transforms with 16-byte loads whose lanes
// cover consecutive bytes, passes them to the owning lanes through shared
// memory padded to an odd row pitch, runs the register DFT, and stores back
// the same way.  Warps work independently (warp-level barriers only).
// ---------------------------------------------------------------------------
template <class RC>
struct RowTrCfg {
    using RC_ = RC;
    using S = typename RC::S;
    static constexpr int N = S::N;
    static constexpr int THREADS = RC::THREADS;
    static constexpr int G = RC::G;
    static constexpr int PITCH = N + 1;
    static constexpr int WARP_FLOATS = 2 * 32 * PITCH;
    static constexpr size_t SMEM = (size_t)(THREADS / 32) * WARP_FLOATS * sizeof(float);
    static_assert(S::T == 1 && S::NS == 1 && N >= 8 && N <= 32, "one thread per transform");
    // (at N = 8 the lanes' own 16-byte rows are already two per 32-byte
    // sector, and this form measured no faster)
    static_assert(THREADS % 32 == 0, "whole warps");
};

template <class CFG, bool ADJ>
__global__ void __launch_bounds__(CFG::THREADS)
k_rows_tr(const float* xr, const float* xi, float* yr, float* yi, long long batch,
          const float2* __restrict__ tw, const W64 w) {
    using S = typename CFG::S;
    constexpr int N = CFG::N, P = CFG::PITCH, Q4 = N / 4;
    constexpr int WARPS = CFG::THREADS / 32;
    extern __shared__ float4 smem4[];
    const int lane = (int)threadIdx.x & 31;
    const int warp = (int)threadIdx.x >> 5;
    float* const t_re = reinterpret_cast<float*>(smem4) + warp * CFG::WARP_FLOATS;
    float* const t_im = t_re + 32 * P;
    const long long groups = (batch + 31) / 32;
    const long long stride = (long long)gridDim.x * WARPS;
    for (long long grp = (long long)blockIdx.x * WARPS + warp; grp < groups; grp += stride) {
        const long long first = grp * 32;
        const int cnt = (int)((batch - first < 32) ? (batch - first) : 32);
        // 32 rows x N floats per plane: N / 4 warp-wide 16-byte loads,
        // float4 q of the block = row q / Q4, columns 4 (q % Q4) .. + 3
        const float4* gr = reinterpret_cast<const float4*>(xr + first * N);
        const float4* gi = reinterpret_cast<const float4*>(xi + first * N);
#pragma unroll
        for (int j = 0; j < Q4; ++j) {
            const int q = lane + 32 * j;
            const int row = q / Q4, c = 4 * (q % Q4);
            if (row < cnt) {
                const float4 a = gr[q];
                const float4 b = gi[q];
                t_re[row * P + c] = a.x; t_re[row * P + c + 1] = a.y;
                t_re[row * P + c + 2] = a.z; t_re[row * P + c + 3] = a.w;
                t_im[row * P + c] = b.x; t_im[row * P + c + 1] = b.y;
                t_im[row * P + c + 2] = b.z; t_im[row * P + c + 3] = b.w;
            }
        }
        __syncwarp();
        float ar[N], ai[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            ar[i] = t_re[lane * P + i];
            ai[i] = t_im[lane * P + i];
        }
        float orr[N], oi[N];
        auto ld = [&](int L, float& r, float& i) { r = ar[L]; i = ai[L]; };
        auto st = [&](int k, float r, float i) { orr[k] = r; oi[k] = i; };
        auto none_w = [](int, float, float) {};
        auto none_r = [](int, float&, float&) {};
        auto twf = [](int, int, int) -> float2 { return make_float2(1.f, 0.f); };
        run_steps<S, ADJ>(0, w, ld, none_w, none_r, twf, st, [] {});
        __syncwarp();   // every lane has read its row before the results overwrite it
#pragma unroll
        for (int k = 0; k < N; ++k) {
            t_re[lane * P + k] = orr[k];
            t_im[lane * P + k] = oi[k];
        }
        __syncwarp();
        float4* yr4 = reinterpret_cast<float4*>(yr + first * N);
        float4* yi4 = reinterpret_cast<float4*>(yi + first * N);
#pragma unroll
        for (int j = 0; j < Q4; ++j) {
            const int q = lane + 32 * j;
            const int row = q / Q4, c = 4 * (q % Q4);
            if (row < cnt) {
                yr4[q] = make_float4(t_re[row * P + c], t_re[row * P + c + 1],
                                     t_re[row * P + c + 2], t_re[row * P + c + 3]);
                yi4[q] = make_float4(t_im[row * P + c], t_im[row * P + c + 1],
                                     t_im[row * P + c + 2], t_im[row * P + c + 3]);
            }
        }
        __syncwarp();   // stores have read the tile before the next group fills it
    }
    (void)tw;
}

template <class CFG>
cudaError_t rows_tr_prepare() {
    if (CFG::SMEM <= 48 * 1024) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_rows_tr<CFG, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CFG::SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_rows_tr<CFG, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)CFG::SMEM);
}

template <class CFG>
int rows_tr_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rows_tr<CFG, false>, CFG::THREADS,
                                                      CFG::SMEM) != cudaSuccess)
        return 0;
    return n;
}

template <class CFG>
cudaError_t rows_tr_launch(const LaunchArgs& a) {
    if (a.adj)
        return launch_kernel(k_rows_tr<CFG, true>, a.grid, CFG::THREADS, CFG::SMEM, a.stream, a.xr,
                             a.xi, a.yr, a.yi, a.batch, a.tw, a.w64);
    return launch_kernel(k_rows_tr<CFG, false>, a.grid, CFG::THREADS, CFG::SMEM, a.stream, a.xr,
                         a.xi, a.yr, a.yi, a.batch, a.tw, a.w64);
}

template <class CFG>
KernelInfo rows_tr_info(const char* name) {
    KernelInfo k = rows_shape<typename CFG::RC_>(name);
    k.smem = CFG::SMEM;
    k.prepare = rows_tr_prepare<CFG>;
    k.blocks_per_sm = rows_tr_blocks_per_sm<CFG>;
    k.launch = rows_tr_launch<CFG>;
    return k;
}

}  // namespace sdft
