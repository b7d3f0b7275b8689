// ragged.cu -- one persistent launch for a batch of mixed power-of-two lengths.
//
// The plan turns the batch into a queue of work items, longest transforms
// first.  Lengths up to 8192 are "row" items: 256 / T transforms of one
// length processed by one 256-thread CTA with the row tile routine.  Lengths
// 16384 .. 65536 are split into pass-1 and pass-2 items (kernels_items.cuh):
// a pass-2 item waits until every pass-1 item of its transform has finished,
// and the pass-1 items of a transform wait until the previous user of its
// scratch slot (a ring of slots sized to stay in L2) has finished pass 2.
// Every dependency points to an item earlier in the queue; the grid is
// persistent (all CTAs resident at once) and CTAs claim items in queue order
// with atomicAdd, so each awaited item is already running and the waits end.
// Each wait is still bounded: past its limit the kernel records
// SDFT_ERR_TIMEOUT in the plan's status word, every later wait returns at
// once, and the kernel runs out its queue and exits.
// The work counter and completion counters are zeroed by a memset node that
// precedes the kernel in the plan's CUDA graph.
#include "../../include/sdft.h"
#include "kernels_items.cuh"
#include "kernels_rows.cuh"
#include "ragged.h"

namespace sdft {
namespace {

constexpr int kThreads = 256;

//                      LOGN LOGE LR0 LR1 LR2    G  SBX
using R2 = RowCfg<2, 2, 2, 0, 0, 256>;
using R3 = RowCfg<3, 3, 3, 0, 0, 256>;
using R4 = RowCfg<4, 4, 4, 0, 0, 256>;
using R5 = RowCfg<5, 5, 5, 0, 0, 256>;
using R6 = RowCfg<6, 3, 3, 3, 0, 32, 2>;
using R7 = RowCfg<7, 4, 4, 3, 0, 32>;
using R8 = RowCfg<8, 4, 4, 4, 0, 16>;
using R9 = RowCfg<9, 5, 5, 4, 0, 16, 16>;
using R10 = RowCfg<10, 5, 5, 5, 0, 8>;
using R11 = RowCfg<11, 5, 5, 4, 2, 4>;
using R12 = RowCfg<12, 5, 5, 5, 2, 2>;
using R13 = RowCfg<13, 5, 5, 5, 3, 1>;
using S256 = Steps<8, 5, 5, 3, 0>;     // 8 threads x 32 values, radix [32,8]
using S128 = Steps<7, 4, 4, 3, 0>;     // 8 threads x 16 values, radix [16,8]
using I14 = ItemCfg<7, 7, S128, S128>;
using I15 = ItemCfg<8, 7, S256, S128>;
using I16 = ItemCfg<8, 8, S256, S256>;

constexpr size_t smax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kSmem =
    smax(smax(smax(R6::SMEM, R7::SMEM), smax(R8::SMEM, R9::SMEM)),
         smax(smax(smax(R10::SMEM, R11::SMEM), smax(R12::SMEM, R13::SMEM)),
              smax(I14::SMEM, smax(I15::SMEM, I16::SMEM))));

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 waits (bounded) until *word >= target; the CTA learns the outcome.
// false: the wait gave up now or an earlier one did (status already set).
__device__ __forceinline__ bool cta_wait(const int* word, int target, const RaggedArgs& a) {
    __shared__ int s_ok;
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

// Publish one finished item: every thread's global writes, then the counter.
__device__ __forceinline__ void cta_signal(int* word) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(word, 1);
    }
}

template <class CFG, bool ADJ>
__device__ __forceinline__ void ragged_rows(const RaggedArgs& a, const int4 item, float* smem) {
    using S = typename CFG::S;
    static_assert(CFG::THREADS == kThreads, "ragged routines use 256 threads");
    const int t = (int)threadIdx.x & (S::T - 1);
    const int g = (int)threadIdx.x >> S::LOGT;
    const bool active = g < item.z;
    const long long row = active ? a.offsets[item.y + g] : 0;
    float* const s_re = smem + g * CFG::BUF;
    float* const s_im = s_re + CFG::PLANE;
    rows_tile<CFG, ADJ>(a.xr + row, a.xi + row, a.yr + row, a.yi + row, active, t, s_re, s_im,
                        a.tw[S::LOGN], a.w);
}

// item.y = long-transform index lt, item.z = tile, item.w = dependency
// (pass 1: the long transform whose pass 2 must free the slot, or -1).
template <class CFG, bool ADJ>
__device__ __forceinline__ void ragged_pass1(const RaggedArgs& a, const int4 item, float* smem) {
    const int lt = item.y;
    if (item.w >= 0 && !cta_wait(a.done2 + item.w, a.tiles2[item.w], a)) return;
    const long long row = a.long_offsets[lt];
    float* const scr = reinterpret_cast<float*>(a.scratch + (size_t)a.long_slot[lt] * a.slot_size);
    item_pass1<CFG, ADJ>(a.xr + row, a.xi + row, scr, scr + CFG::N, item.z, smem, a.tw[CFG::LOGN],
                         a.w);
    cta_signal(a.done1 + lt);
}

template <class CFG, bool ADJ>
__device__ __forceinline__ void ragged_pass2(const RaggedArgs& a, const int4 item, float* smem) {
    const int lt = item.y;
    if (!cta_wait(a.done1 + lt, CFG::TILES1 + a.dep_extra, a)) return;
    const long long row = a.long_offsets[lt];
    const float* scr =
        reinterpret_cast<const float*>(a.scratch + (size_t)a.long_slot[lt] * a.slot_size);
    item_pass2<CFG, ADJ>(scr, scr + CFG::N, a.yr + row, a.yi + row, item.z, smem,
                         a.tw[CFG::LOGN], a.w);
    cta_signal(a.done2 + lt);
}

template <bool ADJ>
__global__ void __launch_bounds__(kThreads, 2) k_ragged(const RaggedArgs a) {
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
            case kPass1 + 14: ragged_pass1<I14, ADJ>(a, item, smem); break;
            case kPass1 + 15: ragged_pass1<I15, ADJ>(a, item, smem); break;
            case kPass1 + 16: ragged_pass1<I16, ADJ>(a, item, smem); break;
            case kPass2 + 14: ragged_pass2<I14, ADJ>(a, item, smem); break;
            case kPass2 + 15: ragged_pass2<I15, ADJ>(a, item, smem); break;
            case kPass2 + 16: ragged_pass2<I16, ADJ>(a, item, smem); break;
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
    c.tiles1 = c.tiles2 = 0;
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
RaggedClass item_class(int logn) {
    using SA = typename CFG::SA_;
    using SC = typename CFG::SC_;
    RaggedClass c = {};
    c.logn = logn;
    c.per_item = 1;
    c.large = true;
    c.tiles1 = CFG::TILES1;
    c.tiles2 = CFG::TILES2;
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
        row_class<R13>(13), item_class<I14>(14), item_class<I15>(15), item_class<I16>(16)};
    return (logn >= 2 && logn <= 16) ? &c[logn] : nullptr;
}

int ragged_threads() { return kThreads; }
size_t ragged_smem() { return kSmem; }
int64_t ragged_slot_size() { return 65536; }

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
