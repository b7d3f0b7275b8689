// ragged.cu -- one persistent launch for a batch of mixed power-of-two lengths.
//
// A ragged plan sorts its transforms by length, largest first, and cuts each
// length class into work items of as many transforms as one 512-thread CTA
// processes at once (512 / T for the row routines, one for N >= 32768).  A
// persistent grid of one CTA per SM claims items from a device counter with
// atomicAdd and runs the routine of the item's length: the same step engine
// and tile routines as the uniform kernels, instantiated for 512 threads.
// Claiming needs no waiting on other CTAs (no spin, no flag), so the launch
// cannot deadlock; the counter is reset to zero by a memset node placed before
// the kernel in the plan's CUDA graph.
#include "kernels_large.cuh"
#include "kernels_rows.cuh"
#include "ragged.h"

namespace sdft {
namespace {

constexpr int kThreads = 512;

//                      LOGN LOGE LR0 LR1 LR2    G  SBX
using R2 = RowCfg<2, 2, 2, 0, 0, 512>;
using R3 = RowCfg<3, 3, 3, 0, 0, 512>;
using R4 = RowCfg<4, 4, 4, 0, 0, 512>;
using R5 = RowCfg<5, 5, 5, 0, 0, 512>;
using R6 = RowCfg<6, 3, 3, 3, 0, 64, 2>;
using R7 = RowCfg<7, 4, 4, 3, 0, 64>;
using R8 = RowCfg<8, 4, 4, 4, 0, 32>;
using R9 = RowCfg<9, 5, 5, 4, 0, 32, 16>;
using R10 = RowCfg<10, 5, 5, 5, 0, 16>;
using R11 = RowCfg<11, 5, 5, 4, 2, 8>;
using R12 = RowCfg<12, 5, 5, 5, 2, 4>;
using R13 = RowCfg<13, 5, 5, 5, 3, 2>;
using R14 = RowCfg<14, 5, 5, 5, 4, 1>;
using S256 = Steps<8, 4, 4, 4, 0>;
using S128 = Steps<7, 4, 4, 3, 0>;
using L15 = LargeCfgT<8, 7, S256, S128>;
using L16 = LargeCfgT<8, 8, S256, S256>;

constexpr size_t smax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kSmem =
    smax(smax(smax(R6::SMEM, R7::SMEM), smax(R8::SMEM, R9::SMEM)),
         smax(smax(smax(R10::SMEM, R11::SMEM), smax(R12::SMEM, R13::SMEM)),
              smax(R14::SMEM, smax(L15::SMEM, L16::SMEM))));

template <class CFG, bool ADJ>
__device__ __forceinline__ void ragged_rows(const RaggedArgs& a, const int4 item, float* smem) {
    using S = typename CFG::S;
    static_assert(CFG::THREADS == kThreads, "ragged routines use 512 threads");
    const int t = (int)threadIdx.x & (S::T - 1);
    const int g = (int)threadIdx.x >> S::LOGT;
    const bool active = g < item.z;
    const long long row = active ? a.offsets[item.y + g] : 0;
    float* const s_re = smem + g * CFG::BUF;
    float* const s_im = s_re + CFG::PLANE;
    rows_tile<CFG, ADJ>(a.xr + row, a.xi + row, a.yr + row, a.yi + row, active, t, s_re, s_im,
                        a.tw[S::LOGN], a.w);
}

template <class CFG, bool ADJ>
__device__ __forceinline__ void ragged_large(const RaggedArgs& a, const int4 item, float* smem) {
    static_assert(CFG::THREADS == kThreads, "ragged routines use 512 threads");
    const long long row = a.offsets[item.y];
    float* const scr_re = reinterpret_cast<float*>(a.scratch + (size_t)blockIdx.x * 65536);
    float* const scr_im = scr_re + CFG::N;
    large_one<CFG, ADJ>(a.xr + row, a.xi + row, a.yr + row, a.yi + row, scr_re, scr_im, smem,
                        a.tw[CFG::LOGN], a.w);
}

template <bool ADJ>
__global__ void __launch_bounds__(kThreads, 1) k_ragged(const RaggedArgs a) {
    extern __shared__ float4 smem4[];
    float* const smem = reinterpret_cast<float*>(smem4);
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();  // every thread has read s_item before it is claimed again
        if (it >= a.nitems) break;
        const int4 item = a.items[it];
        switch (item.x) {
            case 2: ragged_rows<R2, ADJ>(a, item, smem); break;
            case 3: ragged_rows<R3, ADJ>(a, item, smem); break;
            case 4: ragged_rows<R4, ADJ>(a, item, smem); break;
            case 5: ragged_rows<R5, ADJ>(a, item, smem); break;
            case 6: ragged_rows<R6, ADJ>(a, item, smem); break;
            case 7: ragged_rows<R7, ADJ>(a, item, smem); break;
            case 8: ragged_rows<R8, ADJ>(a, item, smem); break;
            case 9: ragged_rows<R9, ADJ>(a, item, smem); break;
            case 10: ragged_rows<R10, ADJ>(a, item, smem); break;
            case 11: ragged_rows<R11, ADJ>(a, item, smem); break;
            case 12: ragged_rows<R12, ADJ>(a, item, smem); break;
            case 13: ragged_rows<R13, ADJ>(a, item, smem); break;
            case 14: ragged_rows<R14, ADJ>(a, item, smem); break;
            case 15: ragged_large<L15, ADJ>(a, item, smem); break;
            case 16: ragged_large<L16, ADJ>(a, item, smem); break;
            default: break;
        }
        // the barrier at the loop top orders the next item's shared-memory
        // writes after every thread's last read of this one
    }
}

template <class CFG>
RaggedClass row_class(int logn) {
    using S = typename CFG::S;
    RaggedClass c = {};
    c.logn = logn;
    c.per_item = CFG::G;
    c.large = false;
    c.ntables = 0;
    if (S::NS > 1) {
        const int64_t n = S::N;
        c.tables[c.ntables++] = TableDesc{n, (int64_t)1 << S::lr(0), n >> S::lr(0), CFG::TW0};
        if (S::NS > 2) {
            const int64_t m1 = n >> S::lr(0);
            c.tables[c.ntables++] = TableDesc{m1, (int64_t)1 << S::lr(1), m1 >> S::lr(1), CFG::TW1};
        }
    }
    c.tw_entries = CFG::TW_TOTAL;
    return c;
}

template <class CFG>
RaggedClass large_class(int logn) {
    using SA = typename CFG::SA_;
    using SC = typename CFG::SC_;
    RaggedClass c = {};
    c.logn = logn;
    c.per_item = 1;
    c.large = true;
    c.ntables = 3;
    c.tables[0] = TableDesc{CFG::A, (int64_t)1 << SA::lr(0), (int64_t)CFG::A >> SA::lr(0), CFG::TWA};
    c.tables[1] = TableDesc{CFG::C, (int64_t)1 << SC::lr(0), (int64_t)CFG::C >> SC::lr(0), CFG::TWC};
    c.tables[2] = TableDesc{CFG::N, CFG::A, CFG::C, CFG::TWB};
    c.tw_entries = CFG::TW_TOTAL;
    return c;
}

}  // namespace

const RaggedClass* ragged_class(int logn) {
    static const RaggedClass c[17] = {
        RaggedClass{}, RaggedClass{}, row_class<R2>(2), row_class<R3>(3), row_class<R4>(4),
        row_class<R5>(5), row_class<R6>(6), row_class<R7>(7), row_class<R8>(8),
        row_class<R9>(9), row_class<R10>(10), row_class<R11>(11), row_class<R12>(12),
        row_class<R13>(13), row_class<R14>(14), large_class<L15>(15), large_class<L16>(16)};
    return (logn >= 2 && logn <= 16) ? &c[logn] : nullptr;
}

int ragged_threads() { return kThreads; }
size_t ragged_smem() { return kSmem; }
int64_t ragged_scratch_per_cta() { return 65536; }

const void* ragged_kernel_fn(bool adj) {
    return adj ? reinterpret_cast<const void*>(k_ragged<true>)
               : reinterpret_cast<const void*>(k_ragged<false>);
}

cudaError_t ragged_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_ragged<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_ragged<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kSmem);
}

int ragged_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ragged<false>, kThreads, kSmem) !=
        cudaSuccess)
        return 0;
    return n;
}

}  // namespace sdft
