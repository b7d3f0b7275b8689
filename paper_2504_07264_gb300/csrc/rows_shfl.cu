// rows_shfl.cu -- short transforms (N = 16 .. 64) spread over L = 2 .. 8
// lanes of a warp, V = N / L contiguous points per lane (8 here).
//
// With n = v + V l (lane l of the transform's L lanes, register v < V) and
// k = kl + L kv, the DFT of Eq. (1) splits into
//   Z[v][kl] = sum_l x[v + V l] W_L^{l kl}                     (step A)
//   X[kl + L kv] = sum_v W_N^{v kl} W_V^{v kv} Z[v][kl]        (step B)
// Step A runs across the lanes: log2 L radix-2 stages in decimation-in-
// frequency order, each a butterfly of the two lanes l and l ^ m exchanged by
// __shfl_xor_sync (the lower lane keeps the sum, the upper one the rotated
// difference, the D(i)/W(i) factors of Eq. (6) applied to a lane pair), which
// leaves Z[v][bitrev(l)] in lane l.  After the rotation by W_N^{v kl}, step B
// is a V-point DFT in registers.  Every lane loads its V inputs and stores
// its V outputs as 16-byte vectors of contiguous bytes; the outputs reach
// their lanes through a small per-warp shared-memory transpose.
#include "fft_core.cuh"
#include "launch.h"
#include "rows_shfl.h"

namespace sdft {
namespace {

template <int LOGN, int LOGV>
struct ShflCfg {
    static constexpr int LOGN_ = LOGN, LOGV_ = LOGV, LOGL = LOGN - LOGV;
    static constexpr int N = 1 << LOGN, V = 1 << LOGV, L = 1 << LOGL;
    static constexpr int TPW = 32 / L;                  // transforms per warp
    static constexpr int THREADS = 256, WARPS = THREADS / 32;
    // transpose row pitch (floats): a multiple of 4 (16-byte reads) with
    // PITCH = L (mod 32) where N is a multiple of 32, so that a warp's writes
    // sub * PITCH + kl fall on 32 banks (two-way for L = 2)
    static constexpr int PITCH = N + (L > 4 ? L : 4);
    static constexpr int WARP_FLOATS = 2 * TPW * PITCH;
    static constexpr size_t SMEM = (size_t)WARPS * WARP_FLOATS * sizeof(float);
    static_assert(L >= 2 && L <= 16 && V >= 4 && V <= 16, "2 .. 16 lanes of 4 .. 16 points");
};

// Twiddle table: W_N^j at tw[N + j], j < N (row 1 of the table [d][j] = W_N^{d j}).
template <class CFG, bool ADJ>
__global__ void __launch_bounds__(256)
k_rows_shfl(const float* xr, const float* xi, float* yr, float* yi, long long batch,
            const float2* __restrict__ tw, const W64 w) {
    constexpr int N = CFG::N, V = CFG::V, L = CFG::L, LOGL = CFG::LOGL, TPW = CFG::TPW;
    constexpr int P = CFG::PITCH;
    extern __shared__ float4 smem4[];
    const int lane = (int)threadIdx.x & 31;
    const int warp = (int)threadIdx.x >> 5;
    float* const t_re = reinterpret_cast<float*>(smem4) + warp * CFG::WARP_FLOATS;
    float* const t_im = t_re + TPW * P;
    const int l = lane & (L - 1);                       // lane within the transform
    const int sub = lane >> LOGL;                       // transform within the warp
    const int kl = (int)(__brev((unsigned)l) >> (32 - LOGL));
    // this lane's rotations: stage s (span m = L >> (s + 1)) multiplies the
    // upper lane's difference by W_{2m}^{l mod m}; step B's input v by W_N^{v kl}
    float2 wst[LOGL > 1 ? LOGL - 1 : 1];
#pragma unroll
    for (int s = 0; s + 1 < LOGL; ++s) {
        const int m = L >> (s + 1);
        wst[s] = (l & m) ? __ldg(tw + N + (l & (m - 1)) * (N / (2 * m))) : make_float2(1.f, 0.f);
    }
    float2 wv[V];
#pragma unroll
    for (int v = 1; v < V; ++v) wv[v] = __ldg(tw + N + (v * kl) % N);
    const long long groups = (batch + TPW - 1) / TPW;
    const long long stride = (long long)gridDim.x * CFG::WARPS;
    for (long long grp = (long long)blockIdx.x * CFG::WARPS + warp; grp < groups; grp += stride) {
        const long long g = grp * TPW + sub;
        const bool active = g < batch;
        float re[V], im[V];
        if (active) {
            const float4* gr = reinterpret_cast<const float4*>(xr + g * N + V * l);
            const float4* gi = reinterpret_cast<const float4*>(xi + g * N + V * l);
#pragma unroll
            for (int q = 0; q < V / 4; ++q) {
                const float4 a = gr[q], b = gi[q];
                re[4 * q] = a.x; re[4 * q + 1] = a.y; re[4 * q + 2] = a.z; re[4 * q + 3] = a.w;
                im[4 * q] = b.x; im[4 * q + 1] = b.y; im[4 * q + 2] = b.z; im[4 * q + 3] = b.w;
            }
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) re[v] = im[v] = 0.f;
        }
        // step A: radix-2 DIF across lanes; lower lane a + b, upper (a - b) W
#pragma unroll
        for (int s = 0; s < LOGL; ++s) {
            const int m = L >> (s + 1);
            const float sg = (l & m) ? -1.f : 1.f;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float pr = __shfl_xor_sync(0xffffffffu, re[v], m);
                const float pi = __shfl_xor_sync(0xffffffffu, im[v], m);
                re[v] = fmaf(sg, re[v], pr);
                im[v] = fmaf(sg, im[v], pi);
                if (m > 1) rot<ADJ>(re[v], im[v], wst[s]);
            }
        }
        // rotation W_N^{v kl}, then step B in registers (output kv in register
        // brevc(kv))
#pragma unroll
        for (int v = 1; v < V; ++v) rot<ADJ>(re[v], im[v], wv[v]);
        dft_regs<V, ADJ>(re, im, 0, w);
        // X[kl + L kv] to row `sub` of the warp's transpose buffer, then each
        // lane takes its V contiguous outputs
        __syncwarp();
#pragma unroll
        for (int kv = 0; kv < V; ++kv) {
            t_re[sub * P + kl + L * kv] = re[brevc(kv, CFG::LOGV_)];
            t_im[sub * P + kl + L * kv] = im[brevc(kv, CFG::LOGV_)];
        }
        __syncwarp();
        if (active) {
            float4* const gr = reinterpret_cast<float4*>(yr + g * N + V * l);
            float4* const gi = reinterpret_cast<float4*>(yi + g * N + V * l);
#pragma unroll
            for (int q = 0; q < V / 4; ++q) {
                gr[q] = *reinterpret_cast<const float4*>(t_re + sub * P + V * l + 4 * q);
                gi[q] = *reinterpret_cast<const float4*>(t_im + sub * P + V * l + 4 * q);
            }
        }
    }
}

template <class CFG>
cudaError_t shfl_prepare() {
    return cudaSuccess;   // shared memory below the 48 KiB default
}

template <class CFG>
int shfl_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_rows_shfl<CFG, false>, CFG::THREADS,
                                                      CFG::SMEM) != cudaSuccess)
        return 0;
    return n;
}

template <class CFG>
cudaError_t shfl_launch(const LaunchArgs& a) {
    if (a.adj)
        return launch_kernel(k_rows_shfl<CFG, true>, a.grid, CFG::THREADS, CFG::SMEM, a.stream,
                             a.xr, a.xi, a.yr, a.yi, a.batch, a.tw, a.w64);
    return launch_kernel(k_rows_shfl<CFG, false>, a.grid, CFG::THREADS, CFG::SMEM, a.stream, a.xr,
                         a.xi, a.yr, a.yi, a.batch, a.tw, a.w64);
}

template <class CFG>
KernelInfo shfl_info(const char* name) {
    static_assert(CFG::SMEM <= 48 * 1024, "default shared-memory limit");
    KernelInfo k = {};
    k.name = name;
    k.logn = CFG::LOGN_;
    k.threads = CFG::THREADS;
    k.smem = CFG::SMEM;
    k.transforms_per_cta = CFG::WARPS * CFG::TPW;
    k.ntables = 1;
    k.tables[0] = TableDesc{CFG::N, 2, CFG::N, 0};     // [d][j] = W_N^{d j}, d < 2
    k.tw_entries = 2 * CFG::N;
    k.scratch_per_cta = 0;
    k.launches = 1;
    k.prepare = shfl_prepare<CFG>;
    k.blocks_per_sm = shfl_blocks_per_sm<CFG>;
    k.launch = shfl_launch<CFG>;
    return k;
}

}  // namespace

const KernelInfo* rows_shfl_candidate(int logn, int idx) {
    // (Measured and left out: N = 8 as 2 x 4 and N = 128 as 16 x 8, no faster
    // than the one-thread and 8-thread forms; N = 128 as 8 lanes x two groups
    // of 8 with a radix-2 step in registers first, 119 registers and slower;
    // N = 16 as 4 x 4, slower than 2 x 8; 16 points per lane, whose 64-byte
    // lane stride halves coalescing.)
    static const KernelInfo k4 = shfl_info<ShflCfg<4, 3>>(
        "N=16: 2 lanes/transform x 8 points, butterflies across lanes by warp shuffles");
    static const KernelInfo k5 = shfl_info<ShflCfg<5, 3>>(
        "N=32: 4 lanes/transform x 8 points, butterflies across lanes by warp shuffles");
    static const KernelInfo k6 = shfl_info<ShflCfg<6, 3>>(
        "N=64: 8 lanes/transform x 8 points, butterflies across lanes by warp shuffles");
    if (idx != 0) return nullptr;
    switch (logn) {
        case 4: return &k4;
        case 5: return &k5;
        case 6: return &k6;
        default: return nullptr;
    }
}

}  // namespace sdft
