// split_tc.cu -- split-precision tensor-core path (SDFT_F32_SPLIT_BF16 and
// SDFT_F32_SPLIT_FP16) for N = 256 and N = 1024.
//
// N = R * R.  A radix-R block of the DFT is a dense real contraction: on the
// stacked planes of R inputs, the R-point DFT is the 2R x 2R real matrix of
// Eqs. (4)-(5), [y^r; y^i] = [C S; -S C] [x^r; x^i] (its transpose for the
// adjoint).  The transform is two such blocks (the regrouping of Eq. (6) into
// radix-R steps used everywhere in this library):
//   GEMM 1: rows (transform b, column c), K = [x^r, x^i](c + R * ntop), ntop < R
//           -> D1[(b, c)][(re/im, d)]                       (tcgen05, TMEM)
//   rotate D1 by W_N^{c * d} in float32
//   GEMM 2: rows (b, d), K = the rotated values over c      (tcgen05, TMEM)
//           -> y[b][d + R * k2]
// Each GEMM runs on 16-bit operands with float32 accumulation: every operand
// is split into hi + lo 16-bit parts (x = hi + lo + O(2^-16 |x|) for bf16) and
// the product is accumulated as hi*B_lo + lo*B_hi + hi*B_hi (the lo*lo term is
// dropped).  For FP16 the input is first scaled by a power of two so that
// the transform's largest magnitude lies in [0.5, 1) (FP16's range and normal
// lo parts); GEMM 1's results are then at most R * sqrt(2) in magnitude, well
// inside FP16's range, and are split as they are; the scale is undone exactly
// at the store.  BF16 has the float32 exponent range, and a power-of-two
// scale would not change its rounding: it is split unscaled.
//
// One CTA of 128 threads (a warpgroup) owns 128 GEMM rows = 128 / R
// transforms per tile; thread i owns row i and TMEM lane i.  Thread 0 issues
// the MMAs (6 per GEMM for R = 16, 12 for R = 32) and commits them to an
// mbarrier.  Data moves in bulk (TMA, 1-D): the block matrices and the
// rotation table W_N^{c d} once per CTA, and each tile's input into shared
// memory (R = 16: the next tile's into a buffer of its own while the current
// one is in its GEMMs; R = 32: into the operand region as soon as GEMM 2 has
// read it).  Outputs leave by one bulk store per plane from shared memory
// (R = 16) or straight from registers, two digits per 8-byte store (R = 32).  Operands
// have no swizzle: 8 x 16-byte core matrices, K-adjacent core matrices 128 B
// apart, M-adjacent ones K/8*128 B apart.  The GEMM-1 operand is K-major:
// thread (b, c) writes its row as 16-byte core-matrix rows.  The GEMM-2
// operand is the GEMM-1 result transposed per transform; it is stored
// MN-major, so that thread (b, c), holding column c of transform b's GEMM-2
// operand after the rotation, writes 8 consecutive rows (b, d) per 16 bytes
// and no float32 transpose is needed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/sdft.h"
#include "fft_core.cuh"
#include "launch.h"
#include "split.h"
#include "tc_ptx.cuh"
#include "twiddle.cuh"

namespace sdft {
namespace {

template <int LOGR, bool FP16>
struct SplitCfg {
    static constexpr int R = 1 << LOGR, N = R * R, LOGN = 2 * LOGR;
    static constexpr int ROWS = 128;            // MMA M
    static constexpr int TPT = ROWS / R;        // transforms per tile
    static constexpr int K = 2 * R;             // [re(0..R-1), im(0..R-1)]
    static constexpr int NM = 2 * R;            // MMA N
    static constexpr int SBO = (K / 8) * 128;   // bytes between 8-row groups
    static constexpr int LBO = 128;             // bytes between K-adjacent core matrices
    static constexpr int A_BYTES = ROWS * K * 2;
    static constexpr int B_BYTES = NM * K * 2;
    static constexpr int TILE_FLOATS = TPT * N;               // one plane of a tile
    static constexpr int X_BYTES = 2 * TILE_FLOATS * 4;       // input tile, both planes
    // R = 16: the next tile's input is prefetched into its own buffer during
    // the GEMMs.  R = 32: the input tile shares the operand region (loaded at
    // the start of each tile), which keeps 4 CTAs per SM within shared memory.
    static constexpr bool PREFETCH = (R == 16);
    // the region holding the GEMM operands (A hi, A lo), then the output tile
    // (and for R = 32 first the input tile)
    static constexpr int AREG_BYTES = 2 * A_BYTES > X_BYTES ? 2 * A_BYTES : X_BYTES;
    static constexpr int TMEM_COLS = 2 * NM;    // D1 and D2 (64 or 128 columns)
    static constexpr int MAX_CTAS = 512 / TMEM_COLS;
    static constexpr int MINB = MAX_CTAS > 4 ? 4 : MAX_CTAS;
    static constexpr uint32_t IDESC = tc::idesc_f16(FP16, ROWS, NM);          // GEMM 1
    static constexpr uint32_t IDESC2 = tc::idesc_f16(FP16, ROWS, NM, true);   // GEMM 2: A MN-major
    // rotation factors W_N^{c d}, d = 1 .. R-1, all c: [d - 1][c]
    static constexpr int TW_BYTES = (R - 1) * R * 8;
    static constexpr int OFF_X = 0, OFF_A = PREFETCH ? X_BYTES : 0, OFF_B = OFF_A + AREG_BYTES;
    static constexpr int OFF_TW = OFF_B + 2 * B_BYTES;
    // x tile, operand region, B hi, B lo, rotation table, plus alignment
    // slack (the base is aligned to 128 bytes); raised so that no more CTAs fit
    // on an SM (228 KiB) than its 512 TMEM columns can serve.
    static constexpr size_t NEED = (size_t)OFF_TW + TW_BYTES + 128;
    static constexpr size_t FLOOR = (size_t)(228 * 1024) / (MAX_CTAS + 1) + 1024;
    static constexpr size_t SMEM = NEED > FLOOR ? NEED : FLOOR;
    static_assert(R == 16 || R == 32, "split path covers N = 256 and 1024");
    static_assert(X_BYTES % 1024 == 0 && AREG_BYTES % 16 == 0 && TW_BYTES % 16 == 0,
                  "alignment");
};

// byte offset of element (row, k) in a K-major, no-swizzle operand
__host__ __device__ constexpr uint32_t kmaj(int row, int k, int sbo) {
    return (uint32_t)((row & 7) * 16 + (row >> 3) * sbo + (k & 7) * 2 + (k >> 3) * 128);
}

// byte offset of elements (rows m .. m + 7, column k), m a multiple of 8, in
// an MN-major, no-swizzle operand with the same core-matrix distances
__host__ __device__ constexpr uint32_t kmn8(int m, int k, int sbo) {
    return (uint32_t)((m >> 3) * sbo + (k >> 3) * 128 + (k & 7) * 16);
}

template <bool FP16>
__device__ __forceinline__ void split16(const float v, uint16_t& hi, uint16_t& lo) {
    if constexpr (FP16) {
        const __half h = __float2half_rn(v);
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(__float2half_rn(v - __half2float(h)));
    } else {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(h)));
    }
}

// Split the pair (a, b) into hi and lo parts, two values per conversion; the
// first value in the low half of each word.  Same rounding as split16.
template <bool FP16>
__device__ __forceinline__ void split16x2(const float a, const float b, uint32_t& hi,
                                          uint32_t& lo) {
    if constexpr (FP16) {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

// Split 8 consecutive values (along K for a K-major operand, along M for an
// MN-major one) into hi and lo parts and store them as one 16-byte
// core-matrix row in each operand.
template <bool FP16>
__device__ __forceinline__ void store_row8(uint8_t* a_hi, uint8_t* a_lo, uint32_t off,
                                           const float* v, float scale) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) split16x2<FP16>(v[2 * j] * scale, v[2 * j + 1] * scale, h[j], l[j]);
    *reinterpret_cast<uint4*>(a_hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(a_lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// D (TMEM columns at dt) = A * B over the three split terms, small terms first.
template <class CFG, uint32_t IDESC>
__device__ __forceinline__ void issue_gemm(uint32_t dt, uint32_t a_hi, uint32_t a_lo,
                                           uint32_t b_hi, uint32_t b_lo) {
    const uint32_t as[3] = {a_hi, a_lo, a_hi};
    const uint32_t bs[3] = {b_lo, b_hi, b_hi};
#pragma unroll
    for (int term = 0; term < 3; ++term)
#pragma unroll
        for (int kk = 0; kk < CFG::K / 16; ++kk) {
            const uint64_t ad = tc::smem_desc(as[term] + kk * 256, CFG::LBO, CFG::SBO);
            const uint64_t bd = tc::smem_desc(bs[term] + kk * 256, CFG::LBO, CFG::SBO);
            tc::mma_f16(dt, ad, bd, IDESC, (term | kk) != 0);
        }
}

// 2R consecutive TMEM columns of this thread's lane
template <int R>
__device__ __forceinline__ void tmem_row(uint32_t taddr, float (&v)[2 * R]) {
    if constexpr (R == 16) {
        tc::tmem_ld32(taddr, v);
    } else {
        float a[32], b[32];
        tc::tmem_ld32(taddr, a);
        tc::tmem_ld32(taddr + 32, b);
#pragma unroll
        for (int i = 0; i < 32; ++i) { v[i] = a[i]; v[32 + i] = b[i]; }
    }
}

template <int R>
__device__ __forceinline__ int block_exponent(const float (&v)[2 * R]) {
    float m = 0.f;
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) m = fmaxf(m, fabsf(v[i]));
#pragma unroll
    for (int o = 1; o < R; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    int e = 0;
    frexpf(m, &e);      // m = f * 2^e, f in [0.5, 1); 0 for m = 0
    return e;
}

// The block exponent used before a split: FP16's, or 0 (no scaling) for BF16.
template <class CFG, int R>
__device__ __forceinline__ int split_exponent(const float (&v)[2 * R]) {
    if constexpr (CFG::FP16_) return block_exponent<R>(v);
    else return 0;
}
template <class CFG>
__device__ __forceinline__ float pow2_scale(const int e) {
    if constexpr (CFG::FP16_) return ldexpf(1.f, e);
    else return 1.f;
}

template <class CFG, bool ADJ>
__global__ void __launch_bounds__(128, CFG::MINB)
k_split(const float* xr, const float* xi, float* yr, float* yi, long long batch,
        const uint16_t* __restrict__ bimg, const float2* __restrict__ tw, int* status) {
    constexpr int R = CFG::R, N = CFG::N, NM = CFG::NM, TPT = CFG::TPT;
    constexpr int TF = CFG::TILE_FLOATS;
    extern __shared__ uint8_t smraw[];
    uint8_t* const sm = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smraw) + 127) & ~static_cast<uintptr_t>(127));
    float* const x_re = reinterpret_cast<float*>(sm + CFG::OFF_X);   // input tile
    float* const x_im = x_re + TF;
    uint8_t* const a_hi = sm + CFG::OFF_A;                            // GEMM operands
    uint8_t* const a_lo = a_hi + CFG::A_BYTES;
    float* const y_re = reinterpret_cast<float*>(sm + CFG::OFF_A);    // output tile (aliases A)
    float* const y_im = y_re + TF;
    uint8_t* const b_hi = sm + CFG::OFF_B;
    const float2* const tw_s = reinterpret_cast<const float2*>(sm + CFG::OFF_TW);
    __shared__ __align__(8) uint64_t mbar[3];
    __shared__ uint32_t tmem_base;
    const int tid = (int)threadIdx.x;
    const int warp = tid >> 5;
    const uint32_t mb_mma = tc::smem_u32(&mbar[0]);
    const uint32_t mb_b = tc::smem_u32(&mbar[1]);
    const uint32_t mb_x = tc::smem_u32(&mbar[2]);
    const uint32_t sa_hi = tc::smem_u32(a_hi), sa_lo = tc::smem_u32(a_lo);
    const uint32_t sb_hi = tc::smem_u32(b_hi), sb_lo = sb_hi + CFG::B_BYTES;

    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&tmem_base), CFG::TMEM_COLS);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(mb_mma, 1);
        tc::mbar_init(mb_b, 1);
        tc::mbar_init(mb_x, 1);
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = tmem_base;
    const uint32_t lane_base = tbase + ((uint32_t)(warp * 32) << 16);

    const long long ntiles = (batch + TPT - 1) / TPT;
    // bulk-load tile `t`'s rows (both planes) into the input buffer
    auto load_tile = [&](long long t) {
        const long long first = t * TPT;
        const long long cnt = (batch - first < TPT) ? (batch - first) : TPT;
        const uint32_t bytes = (uint32_t)(cnt * N * 4);
        tc::mbar_expect_tx(mb_x, 2 * bytes);
        tc::bulk_g2s(tc::smem_u32(x_re), xr + first * N, bytes, mb_x);
        tc::bulk_g2s(tc::smem_u32(x_im), xi + first * N, bytes, mb_x);
    };
    bool x_pending = false;          // thread 0: an input copy not yet waited for
    if (tid == 0) {
        // the block matrices (hi then lo) of this direction and the rotation
        // table, once per CTA
        tc::mbar_expect_tx(mb_b, 2 * CFG::B_BYTES + CFG::TW_BYTES);
        tc::bulk_g2s(sb_hi, bimg + (ADJ ? CFG::B_BYTES : 0), 2 * CFG::B_BYTES, mb_b);
        tc::bulk_g2s(tc::smem_u32(tw_s), tw + R, CFG::TW_BYTES, mb_b);
        if (blockIdx.x < ntiles) { load_tile(blockIdx.x); x_pending = true; }
    }
    int bad = __syncthreads_or(!tc::mbar_wait(mb_b, 0));
    uint32_t ph_mma = 0, ph_x = 0;

    const int bl = tid / R;          // transform within the tile
    const int c = tid % R;           // column (GEMM 1 row) / output digit d (GEMM 2 row)
    for (long long tile = blockIdx.x; !bad && tile < ntiles; tile += gridDim.x) {
        const long long first = tile * TPT;
        const long long cnt = (batch - first < TPT) ? (batch - first) : TPT;
        // R = 16: the previous tile's output store has finished reading the
        // operand region.  (R = 32 stores from registers; its input copy was
        // issued when the previous tile's GEMM 2 completed.)
        if constexpr (CFG::PREFETCH) {
            if (tid == 0) tc::bulk_wait_read0();
        }
        if (__syncthreads_or(!tc::mbar_wait(mb_x, ph_x))) { bad = 1; break; }
        ph_x ^= 1;
        x_pending = false;
        // ---- GEMM 1 operand: row (b, c) = x[c + R * ntop], scaled and split
        float v[2 * R];
#pragma unroll
        for (int t = 0; t < R; ++t) {
            v[t] = x_re[bl * N + c + R * t];
            v[R + t] = x_im[bl * N + c + R * t];
        }
        const int e0 = split_exponent<CFG, R>(v);
        const float s0 = pow2_scale<CFG>(-e0);
        if constexpr (!CFG::PREFETCH) __syncthreads();   // input read before the operands overwrite it
#pragma unroll
        for (int k8 = 0; k8 < 2 * R / 8; ++k8)
            store_row8<CFG::FP16_>(a_hi, a_lo, kmaj(tid, 8 * k8, CFG::SBO), v + 8 * k8, s0);
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            issue_gemm<CFG, CFG::IDESC>(tbase, sa_hi, sa_lo, sb_hi, sb_lo);
            tc::mma_commit(mb_mma);
            if (CFG::PREFETCH && tile + gridDim.x < ntiles) {              // prefetch
                load_tile(tile + gridDim.x);
                x_pending = true;
            }
        }
        if (__syncthreads_or(!tc::mbar_wait(mb_mma, ph_mma))) { bad = 1; break; }
        ph_mma ^= 1;
        tc::fence_after_sync();
        // ---- rotate row (b, c) by W_N^{c d}: column c (re) and R + c (im) of
        // transform b's GEMM-2 operand, rows (b, d), stored MN-major (GEMM 1
        // has finished reading the operand region)
        float d1[2 * R];
        tmem_row<R>(lane_base, d1);
        {
            // W_N^{c d} = W_N^{c d0} W_N^{c A0 d1} (d = d0 + A0 d1): the table's rows
            // below A0 and at the multiples of A0 (R = 32: 10 loads and 21 products
            // instead of 31 loads; R = 16: 6 and 9 instead of 15; one rounding more)
            constexpr int A0 = R == 32 ? 8 : 4, B0 = R / A0;
            float2 wa[A0], wb[B0];
#pragma unroll
            for (int q = 1; q < A0; ++q) wa[q] = tw_s[(q - 1) * R + c];
#pragma unroll
            for (int q = 1; q < B0; ++q) wb[q] = tw_s[(A0 * q - 1) * R + c];
#pragma unroll
            for (int d = 1; d < R; ++d) {
                const int d0 = d % A0, dq = d / A0;
                float2 wv;
                if (dq == 0) wv = wa[d0];
                else if (d0 == 0) wv = wb[dq];
                else wv = make_float2(wa[d0].x * wb[dq].x - wa[d0].y * wb[dq].y,
                                      wa[d0].x * wb[dq].y + wa[d0].y * wb[dq].x);
                rot<ADJ>(d1[d], d1[R + d], wv);
            }
        }
#pragma unroll
        for (int j = 0; j < R / 8; ++j) {
            store_row8<CFG::FP16_>(a_hi, a_lo, kmn8(bl * R + 8 * j, c, CFG::SBO), d1 + 8 * j, 1.f);
            store_row8<CFG::FP16_>(a_hi, a_lo, kmn8(bl * R + 8 * j, R + c, CFG::SBO),
                                   d1 + R + 8 * j, 1.f);
        }
        tc::fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            issue_gemm<CFG, CFG::IDESC2>(tbase + NM, sa_hi, sa_lo, sb_hi, sb_lo);
            tc::mma_commit(mb_mma);
        }
        if (__syncthreads_or(!tc::mbar_wait(mb_mma, ph_mma))) { bad = 1; break; }
        ph_mma ^= 1;
        tc::fence_after_sync();
        const float us = pow2_scale<CFG>(e0);
        float d2[2 * R];
        if constexpr (!CFG::PREFETCH) {
            // R = 32: GEMM 2 has read the operand region, nothing else will:
            // the next tile's input copy starts now, overlapping this tile's
            // TMEM reads and stores.  (An L2 prefetch of the tile after it as
            // well measured 361 against 376 Gpts/s for BF16: the extra lines
            // compete for L2 with the copies and stores in flight.)
            if (tid == 0 && tile + gridDim.x < ntiles) {
                load_tile(tile + gridDim.x);
                x_pending = true;
            }
            // ---- row (b, d): y[d + R * k2] for every k2, scales undone, straight
            // from registers.  A warp holds one transform's 32 digits d; lanes
            // c and c ^ 1 trade values so that each stores two consecutive
            // digits of every other k2 as one 8-byte store (each half-warp's
            // store is one whole 128-byte line): half the store instructions
            // of one value per lane, which fill the memory-instruction queue
            tmem_row<R>(lane_base + NM, d2);
            tc::fence_before_sync();
            {
                const bool odd = (c & 1) != 0;
                float* const gyr = yr + (first + bl) * N + (c & ~1);
                float* const gyi = yi + (first + bl) * N + (c & ~1);
#pragma unroll
                for (int k = 0; k < R; k += 2) {
                    // the even lane keeps k2 = k and sends k + 1, the odd one the reverse
                    const float sr = odd ? d2[k] : d2[k + 1];
                    const float si = odd ? d2[R + k] : d2[R + k + 1];
                    const float rr = __shfl_xor_sync(0xffffffffu, sr, 1);
                    const float ri = __shfl_xor_sync(0xffffffffu, si, 1);
                    if (bl < cnt) {   // the same for the whole warp (one transform)
                        if (!odd) {
                            *reinterpret_cast<float2*>(gyr + R * k) = make_float2(d2[k] * us, rr * us);
                            *reinterpret_cast<float2*>(gyi + R * k) =
                                make_float2(d2[R + k] * us, ri * us);
                        } else {
                            *reinterpret_cast<float2*>(gyr + R * (k + 1)) =
                                make_float2(rr * us, d2[k + 1] * us);
                            *reinterpret_cast<float2*>(gyi + R * (k + 1)) =
                                make_float2(ri * us, d2[R + k + 1] * us);
                        }
                    }
                }
            }
        } else {
            // ---- row (b, d): y[d + R * k2] for every k2, scales undone, via a
            // shared output tile and one bulk store per plane
            tmem_row<R>(lane_base + NM, d2);
            tc::fence_before_sync();
#pragma unroll
            for (int k2 = 0; k2 < R; ++k2) {
                y_re[bl * N + c + R * k2] = d2[k2] * us;
                y_im[bl * N + c + R * k2] = d2[R + k2] * us;
            }
            tc::fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                const uint32_t bytes = (uint32_t)(cnt * N * 4);
                tc::bulk_s2g(yr + first * N, tc::smem_u32(y_re), bytes);
                tc::bulk_s2g(yi + first * N, tc::smem_u32(y_im), bytes);
                tc::bulk_commit();
            }
        }
    }
    if (tid == 0) {
        tc::bulk_wait0();                          // output stores complete
        if (x_pending) tc::mbar_wait(mb_x, ph_x);  // no input copy left in flight (bounded)
        if (bad) atomicExch(status, SDFT_ERR_TIMEOUT);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, CFG::TMEM_COLS);
    }
}

template <int LOGR, bool FP16>
struct SplitCfgT : SplitCfg<LOGR, FP16> {
    static constexpr bool FP16_ = FP16;
};

// Block-matrix images, forward then adjoint, each hi then lo, laid out exactly
// as the kernel's shared-memory B operand: row n = output (re d | im d),
// column k = input (re t | im t).
template <class CFG>
__global__ void k_bimg(uint16_t* dst) {
    constexpr int R = CFG::R;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= 2 * CFG::NM * CFG::K) return;
    const bool adj = u >= CFG::NM * CFG::K;
    const int nk = u % (CFG::NM * CFG::K);
    const int n = nk / CFG::K, k = nk % CFG::K;
    const int d = n % R, t = k % R;
    const float2 w = twiddle_value((int64_t)((d * t) % R), R);   // (cos, -sin) of 2 pi d t / R
    const float cs = w.x, sn = adj ? w.y : -w.y;                  // sin for the forward
    float coef;
    if (n < R) coef = (k < R) ? cs : sn;     // y^r = C x^r + S x^i
    else coef = (k < R) ? -sn : cs;          // y^i = -S x^r + C x^i
    uint16_t h, l;
    split16<CFG::FP16_>(coef, h, l);
    const uint32_t o = kmaj(n, k, CFG::SBO) / 2;
    uint16_t* img = dst + (adj ? 2 * CFG::B_BYTES / 2 : 0);
    img[o] = h;
    img[CFG::B_BYTES / 2 + o] = l;
}

// Dynamic shared memory, and the largest shared-memory carveout (N = 1024
// needs all 228 KiB of an SM for 4 CTAs).
template <class CFG>
cudaError_t split_prepare() {
    for (const void* f : {(const void*)k_split<CFG, false>, (const void*)k_split<CFG, true>}) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)CFG::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Resident CTAs per SM.  The runtime's occupancy query answers 1 for these
// TMEM-allocating kernels although registers and shared memory allow more,
// so the bound is computed from the kernel's own footprint: registers (per
// warp, in units of 256), shared memory (plus the 1 KiB the CUDA runtime reserves
// per CTA), warps, and the SM's 512 TMEM columns.
template <class CFG>
int split_blocks_per_sm() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_split<CFG, false>);
    if (e != cudaSuccess) return -(int)e;
    int dev = 0, regs = 0, smem = 0, warps = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&warps, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) != cudaSuccess)
        return -(int)e;
    const int regs_per_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    int n = regs / (regs_per_warp * 4);
    const int smem_cta = (int)(fa.sharedSizeBytes + CFG::SMEM) + 1024;
    n = n < smem / smem_cta ? n : smem / smem_cta;
    n = n < (warps / 32) / 4 ? n : (warps / 32) / 4;
    return n < CFG::MAX_CTAS ? n : CFG::MAX_CTAS;
}

template <class CFG>
cudaError_t split_launch(const LaunchArgs& a) {
    const uint16_t* bimg = static_cast<const uint16_t*>(a.aux);
    if (a.adj)
        return launch_kernel(k_split<CFG, true>, a.grid, 128, CFG::SMEM, a.stream, a.xr, a.xi, a.yr,
                             a.yi, a.batch, bimg, a.tw, a.status);
    return launch_kernel(k_split<CFG, false>, a.grid, 128, CFG::SMEM, a.stream, a.xr, a.xi, a.yr,
                         a.yi, a.batch, bimg, a.tw, a.status);
}

template <class CFG>
cudaError_t split_make_aux(void* dst, cudaStream_t stream) {
    const int total = 2 * CFG::NM * CFG::K;
    return launch_kernel(k_bimg<CFG>, (total + 255) / 256, 256, 0, stream,
                         static_cast<uint16_t*>(dst));
}

template <class CFG>
SplitInfo split_info(const char* name) {
    SplitInfo s = {};
    KernelInfo& k = s.kern;
    k.name = name;
    k.logn = CFG::LOGN;
    k.threads = 128;
    k.smem = CFG::SMEM;
    k.transforms_per_cta = CFG::TPT;
    k.ntables = 1;
    k.tables[0] = TableDesc{CFG::N, CFG::R, CFG::R, 0};   // W_N^{c d} at [d][c]
    k.tw_entries = CFG::N;
    k.scratch_per_cta = 0;
    k.launches = 1;
    k.prepare = split_prepare<CFG>;
    k.blocks_per_sm = split_blocks_per_sm<CFG>;
    k.launch = split_launch<CFG>;
    s.aux_bytes = 4 * (size_t)CFG::B_BYTES;
    s.make_aux = split_make_aux<CFG>;
    return s;
}

}  // namespace

const SplitInfo* split_kernel(int logn, int dtype) {
    static const SplitInfo b8 = split_info<SplitCfgT<4, false>>(
        "N=256 split-BF16 tensor cores: two 128x32x32 tcgen05 GEMMs (3 terms each) per 8 transforms");
    static const SplitInfo h8 = split_info<SplitCfgT<4, true>>(
        "N=256 split-FP16 tensor cores: two 128x32x32 tcgen05 GEMMs (3 terms each) per 8 transforms");
    static const SplitInfo b10 = split_info<SplitCfgT<5, false>>(
        "N=1024 split-BF16 tensor cores: two 128x64x64 tcgen05 GEMMs (3 terms each) per 4 transforms");
    static const SplitInfo h10 = split_info<SplitCfgT<5, true>>(
        "N=1024 split-FP16 tensor cores: two 128x64x64 tcgen05 GEMMs (3 terms each) per 4 transforms");
    const bool fp16 = dtype == SDFT_F32_SPLIT_FP16;
    if (logn == 8) return fp16 ? &h8 : &b8;
    if (logn == 10) return fp16 ? &h10 : &b10;
    return nullptr;
}

}  // namespace sdft
