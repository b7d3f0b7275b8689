// ragged.cu -- one persistent launch for a batch of mixed power-of-two lengths.
//
// The kernel runs as thread-block clusters of 8 CTAs (256 threads each, two
// per SM).  The plan turns the batch into a queue of cluster items, longest
// transforms first, and each cluster claims one item at a time with an
// atomicAdd by its first CTA, broadcast to the others through distributed
// shared memory and a cluster barrier (each item claims the next one while
// it runs; during a long item the claim rides on the item's own barriers):
//   * a long item (N = 16384 .. 65536) is one, two or four transforms, each
//     held by 8, 4 or 2 CTAs of the cluster in their shared memory and
//     transformed in two passes with the exchange between them done by
//     ld.shared::cluster (kernels_cluster.cuh) -- no global scratch, no
//     inter-CTA waits;
//   * a row item group (N <= 8192) is up to eight row items, one per CTA,
//     each a tile of transforms of one length run by the row tile routine.
// A transform is computed with the same arithmetic and tables as the uniform
// kernel of its length (the cluster kernel for long lengths).
// The work counter is zeroed by a memset node that precedes the kernel in the
// plan's CUDA graph.  The kernel has no device-side waits of its own; for
// tests, a plan can make every long item first wait for a word that nothing
// sets, a wait bounded like all others: past its limit it records
// SDFT_ERR_TIMEOUT in the status word and the item proceeds.
#include "../../include/sdft.h"
#include "kernels_cluster.cuh"
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
// the same radix splits with the register DFTs in the order of Eq. (6); a
// plan picks one of the two per length (RaggedArgs::alt, set by
// sdft_plan_ragged_autotune)
using R5D = RowCfg<5, 5, 5, 0, 0, 256, 0, 1, true>;
using R6D = RowCfg<6, 3, 3, 3, 0, 32, 2, 1, true>;
using R7D = RowCfg<7, 4, 4, 3, 0, 32, 0, 1, true>;
using R8D = RowCfg<8, 4, 4, 4, 0, 16, 0, 1, true>;
using R9D = RowCfg<9, 5, 5, 4, 0, 16, 16, 1, true>;
using R10D = RowCfg<10, 5, 5, 5, 0, 8, 0, 1, true>;
using R11D = RowCfg<11, 5, 5, 4, 2, 4, 0, 1, true>;
using R12D = RowCfg<12, 5, 5, 5, 2, 2, 0, 1, true>;
using R13D = RowCfg<13, 5, 5, 5, 3, 1, 0, 1, true>;

constexpr size_t smax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kSmem =
    smax(smax(smax(R6::SMEM, R7::SMEM), smax(R8::SMEM, R9::SMEM)),
         smax(smax(smax(R10::SMEM, R11::SMEM), smax(R12::SMEM, R13::SMEM)),
              smax(Cluster14::SMEM, smax(Cluster15::SMEM, Cluster16::SMEM))));

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

// Work records.  The cluster's first thread claims a cluster item and writes
// into every CTA's slot that CTA's share of it (st.shared::cluster), so no
// CTA needs a dependent global load to start:
//   x < 0                end of the queue
//   x = kIdle            nothing for this CTA (row groups of fewer than 8)
//   x = 2 .. 13          the row item itself (log2 N, first, count)
//   x = kLong + log2 N   long item: y = 1 if this CTA holds a transform, whose
//                        row start (floats) is z | w << 32
// Two slots alternate, so a slot is rewritten only after every CTA has passed
// a cluster barrier that follows its read.
constexpr int kIdle = 1;

__device__ __forceinline__ void st_cluster4(uint32_t addr, int4 v) {
    asm volatile("st.shared::cluster.v4.b32 [%0], {%1, %2, %3, %4};"
                 :: "r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}

__device__ __forceinline__ int4 load_citem(const RaggedArgs& a, int it) {
    return it < a.nitems ? a.citems[it] : make_int4(-1, 0, 0, 0);
}

// Leader: the records of cluster item `ci` for every CTA, into `slot`.
__device__ __forceinline__ void publish_work(const RaggedArgs& a, const int4 ci, int4* slot) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(slot);
    int4 rec[kRaggedCluster];
    if (ci.x < 0) {
#pragma unroll
        for (int r = 0; r < kRaggedCluster; ++r) rec[r] = make_int4(-1, 0, 0, 0);
    } else if (ci.x >= kLong) {
        const int lq = ci.x - kLong - 13;    // log2 of the CTAs per transform
#pragma unroll
        for (int r = 0; r < kRaggedCluster; ++r) {
            const int sub = r >> lq;
            if (sub < ci.z) {
                const long long off = a.long_offsets[ci.y + sub];
                rec[r] = make_int4(ci.x, 1, (int)(uint32_t)off, (int)(uint32_t)(off >> 32));
            } else {
                rec[r] = make_int4(ci.x, 0, 0, 0);
            }
        }
    } else {
#pragma unroll
        for (int r = 0; r < kRaggedCluster; ++r)
            rec[r] = r < ci.z ? a.items[ci.y + r] : make_int4(kIdle, 0, 0, 0);
    }
#pragma unroll
    for (int r = 0; r < kRaggedCluster; ++r) st_cluster4(map_rank(s, (uint32_t)r), rec[r]);
}

// A long item: this CTA's share (rank q of the Q holding transform `sub`).
// CTAs without a transform take the two cluster barriers only.  The
// cluster's first thread claims the next item meanwhile and publishes its
// records into `next` before the first barrier, so the next item starts
// without a claim barrier of its own.
template <class CFG, bool ADJ>
__device__ __forceinline__ void ragged_long(const RaggedArgs& a, const int4 rec, float* smem,
                                            const uint32_t rank, int4* next) {
    constexpr int Q = CFG::Q, A = CFG::A, C = CFG::C;
    const int tid = (int)threadIdx.x;
    const bool leader = rank == 0 && tid == 0;
    const uint32_t sub = rank / Q, q = rank % Q;
    int claim = 0;
    if (leader) claim = atomicAdd(a.counter, 1);
    if (a.inject) cta_wait(a.never, 1, a);
    if (rec.y == 0) {         // never the leader's CTA: a long item holds >= 1 transform
        cluster_arrive();     // the barrier after pass 1
        cluster_wait();
        cluster_arrive();     // the barrier inside pass 2
        cluster_wait();
        return;
    }
    const long long off = (long long)(((uint64_t)(uint32_t)rec.w << 32) | (uint32_t)rec.z);
    const float2* tw = a.tw[CFG::LOGN];
    const int col = (int)q * CFG::CQ + tid % CFG::CQ;
    const int d = (int)q * CFG::AQ + tid % CFG::AQ;
    const float* gxr = a.xr + off;
    const float* gxi = a.xi + off;
    auto ld = [&](int L, float& r, float& i) {
        r = gxr[col + C * L];
        i = gxi[col + C * L];
    };
    int4 nci = make_int4(-1, 0, 0, 0);
    auto mid = [&] {
        if (leader) nci = load_citem(a, claim);
    };
    pass1<CFG, ADJ>(ld, mid, smem, tid, col, tw, a.w);
    if (leader) publish_work(a, nci, next);
    cluster_arrive();
    cluster_wait();
    float* const gyr = a.yr + off;
    float* const gyi = a.yi + off;
    auto st = [&](int k2, float r, float i) {
        gyr[d + A * k2] = r;
        gyi[d + A * k2] = i;
    };
    pass2<CFG, ADJ>(st, smem, (uint32_t)__cvta_generic_to_shared(smem), tid, d, sub * Q, tw, a.w);
}

template <bool ADJ>
__global__ void __launch_bounds__(kThreads, 2) k_ragged(const RaggedArgs a) {
    extern __shared__ float4 smem4[];
    float* const smem = reinterpret_cast<float*>(smem4);
    __shared__ __align__(16) int4 s_work[2];
    const uint32_t rank = cluster_ctarank();
    const bool leader = rank == 0 && threadIdx.x == 0;
    // every CTA of the cluster is running before any shared memory of it is
    // written from another CTA; then the first item's records
    cluster_arrive();
    cluster_wait();
    if (leader) publish_work(a, load_citem(a, atomicAdd(a.counter, 1)), &s_work[0]);
    cluster_arrive();
    cluster_wait();
    // Each item publishes the records of the next one into the other slot
    // before a cluster barrier: a long item before its own first barrier, a
    // row group at its end, followed by a barrier that also lets the next
    // item reuse every CTA's shared memory.
    for (int par = 0;; par ^= 1) {
        const int4 rec = s_work[par];
        if (rec.x < 0) break;
        int4* const next = &s_work[par ^ 1];
        if (rec.x >= kLong) {
            switch (rec.x - kLong) {
                case 14: ragged_long<Cluster14, ADJ>(a, rec, smem, rank, next); break;
                case 15: ragged_long<Cluster15, ADJ>(a, rec, smem, rank, next); break;
                case 16: ragged_long<Cluster16, ADJ>(a, rec, smem, rank, next); break;
                default: break;
            }
            continue;
        }
        int claim = 0;
        if (leader) claim = atomicAdd(a.counter, 1);
        const bool alt = (a.alt >> rec.x) & 1u;
        switch (rec.x) {
            case 2: ragged_rows<R2, ADJ>(a, rec, smem); break;
            case 3: ragged_rows<R3, ADJ>(a, rec, smem); break;
            case 4: ragged_rows<R4, ADJ>(a, rec, smem); break;
            case 5:
                if (alt) ragged_rows<R5D, ADJ>(a, rec, smem);
                else ragged_rows<R5, ADJ>(a, rec, smem);
                break;
            case 6:
                if (alt) ragged_rows<R6D, ADJ>(a, rec, smem);
                else ragged_rows<R6, ADJ>(a, rec, smem);
                break;
            case 7:
                if (alt) ragged_rows<R7D, ADJ>(a, rec, smem);
                else ragged_rows<R7, ADJ>(a, rec, smem);
                break;
            case 8:
                if (alt) ragged_rows<R8D, ADJ>(a, rec, smem);
                else ragged_rows<R8, ADJ>(a, rec, smem);
                break;
            case 9:
                if (alt) ragged_rows<R9D, ADJ>(a, rec, smem);
                else ragged_rows<R9, ADJ>(a, rec, smem);
                break;
            case 10:
                if (alt) ragged_rows<R10D, ADJ>(a, rec, smem);
                else ragged_rows<R10, ADJ>(a, rec, smem);
                break;
            case 11:
                if (alt) ragged_rows<R11D, ADJ>(a, rec, smem);
                else ragged_rows<R11, ADJ>(a, rec, smem);
                break;
            case 12:
                if (alt) ragged_rows<R12D, ADJ>(a, rec, smem);
                else ragged_rows<R12, ADJ>(a, rec, smem);
                break;
            case 13:
                if (alt) ragged_rows<R13D, ADJ>(a, rec, smem);
                else ragged_rows<R13, ADJ>(a, rec, smem);
                break;
            default: break;   // kIdle
        }
        if (leader) publish_work(a, load_citem(a, claim), next);
        cluster_arrive();
        cluster_wait();
    }
}

template <class CFG>
RaggedClass row_class(int logn) {
    RaggedClass c = {};
    c.logn = logn;
    c.per_item = CFG::G;
    c.large = false;
    c.ntables = rows_tables<CFG>(c.tables);
    c.tw_entries = CFG::TW_TOTAL;
    return c;
}

template <class CFG>
RaggedClass long_class(int logn) {
    using SA = typename CFG::SA_;
    using SC = typename CFG::SC_;
    RaggedClass c = {};
    c.logn = logn;
    c.per_item = kRaggedCluster / CFG::Q;
    c.large = true;
    c.ntables = 4;
    c.tables[0] = TableDesc{CFG::A, (int64_t)1 << SA::lr(0), (int64_t)CFG::A >> SA::lr(0), CFG::TWA};
    c.tables[1] = TableDesc{CFG::C, (int64_t)1 << SC::lr(0), (int64_t)CFG::C >> SC::lr(0), CFG::TWC};
    c.tables[2] = TableDesc{CFG::N, CFG::P, CFG::C, CFG::TWB1};
    c.tables[3] = TableDesc{CFG::N / CFG::P, CFG::R1, CFG::C, CFG::TWB2};
    c.tw_entries = CFG::TW_TOTAL;
    return c;
}

}  // namespace

// log2 N of the classes with an alternative routine
unsigned ragged_alt_classes() { return 0x3FE0u; }   // 5 .. 13

const RaggedClass* ragged_class(int logn) {
    static const RaggedClass c[17] = {
        RaggedClass{}, RaggedClass{}, row_class<R2>(2), row_class<R3>(3), row_class<R4>(4),
        row_class<R5>(5), row_class<R6>(6), row_class<R7>(7), row_class<R8>(8),
        row_class<R9>(9), row_class<R10>(10), row_class<R11>(11), row_class<R12>(12),
        row_class<R13>(13), long_class<Cluster14>(14), long_class<Cluster15>(15),
        long_class<Cluster16>(16)};
    return (logn >= 2 && logn <= 16) ? &c[logn] : nullptr;
}

int ragged_threads() { return kThreads; }
size_t ragged_smem() { return kSmem; }

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

int ragged_resident_ctas() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(kRaggedCluster * 2 * sms), 1, 1);
    cfg.blockDim = dim3((unsigned)kThreads, 1, 1);
    cfg.dynamicSmemBytes = kSmem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kRaggedCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_ragged<false>, &cfg) != cudaSuccess) return 0;
    return clusters * kRaggedCluster;
}

}  // namespace sdft
