// sdft_api.cu -- the C ABI declared in include/sdft.h: plan lifecycle,
// argument validation, kernel dispatch and the host-buffer path.
//
// All validation happens on the host before anything is enqueued, so a bad
// call never reaches the GPU.  Plans are tracked in a registry, so a NULL,
// destroyed or foreign handle is rejected without being dereferenced.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <mutex>
#include <new>
#include <set>
#include <utility>
#include <vector>

#include "../../include/sdft.h"
#include <nvtx3/nvToolsExt.h>

#include "launch.h"
#include "ragged.h"
#include "split.h"

namespace sdft {
const KernelInfo* rows_candidate_small(int logn, int idx);
const KernelInfo* rows_candidate_1024(int logn, int idx);
const KernelInfo* rows_candidate_big(int logn, int idx);
const KernelInfo* rows_pf_candidate(int logn, int idx);
const KernelInfo* rows_candidate_e64(int logn, int idx);

// The work-queue schedule of a long length: the persistent kernel of ragged
// plans (ragged.cu) on a uniform batch, with the length's selected form.
const KernelInfo* queue_candidate(int logn) {
    static KernelInfo q[17];
    static const bool init = [] {
        static const char* names[17] = {};
        names[14] = "N=16384: work queue of the persistent ragged kernel (clusters of 8 CTAs)";
        names[15] = "N=32768: work queue of the persistent ragged kernel (clusters of 8 CTAs)";
        names[16] = "N=65536: work queue of the persistent ragged kernel (clusters of 8 CTAs)";
        for (int l = 14; l <= 16; ++l) {
            q[l] = KernelInfo{};
            q[l].name = names[l];
            q[l].logn = l;
            q[l].threads = 128;
            q[l].transforms_per_cta = 1;
            q[l].launches = 1;
            q[l].queue = true;
        }
        return true;
    }();
    (void)init;
    return (logn >= 14 && logn <= 16) ? &q[logn] : nullptr;
}

// Compiled FP32 schedule `idx` for log2 N (null past the last one).
const KernelInfo* f32_candidate(int logn, int idx) {
    if (logn >= 1 && logn <= 8) return rows_candidate_small(logn, idx);
    if (logn == 10) return rows_candidate_1024(logn, idx);
    if (logn == 9 || logn == 11 || logn == 12) {
        const auto base = logn == 9 ? rows_candidate_small : rows_candidate_big;
        const KernelInfo* k = base(logn, idx);
        if (k) return k;
        int n = 0;
        while (base(logn, n)) ++n;
        return idx >= n ? rows_pf_candidate(logn, idx - n) : nullptr;
    }
    if (logn == 13) {
        int n = 0, m = 0;
        while (rows_candidate_big(logn, n)) ++n;
        while (rows_pf_candidate(logn, m)) ++m;
        if (idx < n) return rows_candidate_big(logn, idx);
        if (idx < n + m) return rows_pf_candidate(logn, idx - n);
        return rows_candidate_e64(logn, idx - n - m);
    }
    if (logn == 14) {
        const KernelInfo* k = rows_candidate_big(logn, idx);
        if (k) return k;
        int n = 0;
        while (rows_candidate_big(logn, n)) ++n;
        if (idx == n) return queue_candidate(14);
        if (idx == n + 1) return cluster_kernel(14, 0);
        if (idx == n + 2) return rows_pf_candidate(14, 0);
        if (idx == n + 3) return cluster_kernel(14, 1);
        return idx == n + 4 ? rows_pf_candidate(14, 1) : nullptr;
    }
    if (logn >= 15 && logn <= 16) {
        if (idx == 0) return queue_candidate(logn);
        if (idx == 1) return large_kernel(logn);
        if (idx >= 2) return cluster_kernel(logn, idx - 2);
    }
    return nullptr;
}

const KernelInfo* rows_kernel(int logn) { return f32_candidate(logn, 0); }
}  // namespace sdft

using namespace sdft;

namespace {

constexpr uint64_t kMagic = 0x53444654504c414eull;  // "SDFTPLAN"
constexpr int kMaxLogN = 16;

thread_local int g_last_error = SDFT_OK;

// NVTX range around an entry point (visible in Nsight tools; a no-op otherwise)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

int fail(int status) {
    g_last_error = status;
    return status;
}

struct HostStaging {
    int mode = 0;                      // SDFT_HOST_AUTO / _STAGED / _ZERO_COPY
    int64_t chunk = 0;                 // transforms per chunk
    float* d_buf[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [slot][plane]
    cudaStream_t streams[2] = {nullptr, nullptr};
    cudaEvent_t start = nullptr;
    float2* d_scratch = nullptr;       // second scratch set for the second slot
};

// State of a ragged plan: the form of every length class, the work items of
// each phase and one CUDA graph per direction (a memset of the claim
// counters, then the persistent kernel).
struct RaggedState {
    bool on = false;
    bool uniform = false;             // a uniform batch of long transforms
    int64_t count = 0;
    std::vector<signed char> logn;    // log2 N of every transform, caller's order
    std::vector<long long> start;     // row start (floats) of every transform
    int form[17] = {};                // form of every length class
    unsigned classes = 0;             // bit l set: some transform has log2 N = l
    const float2* rtw[kRaggedRoutines] = {};   // twiddle tables of every routine
    int4* d_items[kRaggedPhases] = {};         // capacity `count` each
    int nitems[kRaggedPhases] = {};
    long long* d_offsets = nullptr;    // row items: row starts in work order
    int* d_sync = nullptr;             // [claim counters of the phases, a word that stays zero]
    int wait_polls = 1 << 23;          // bound of every device-side wait (polls)
    int inject = 0;                    // tests: group items wait for a word nothing sets
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaGraphNode_t knode[2] = {nullptr, nullptr};
    RaggedArgs args[2] = {};
    std::mutex mu;
};

}  // namespace

struct sdft_plan {
    uint64_t magic;
    int device;
    int dtype;
    int64_t n;            // 0 for ragged plans
    int64_t batch;
    int64_t points;
    const KernelInfo* kern;
    int grid;
    int occupancy;        // CTAs per SM from the occupancy query (negative: its error)
    float2* d_tw;
    float2* d_scratch;
    int* d_status;
    void* d_aux;          // split path: block-matrix images
    W64 w64;
    HostStaging host;
    RaggedState rag;
};

namespace {

std::mutex g_registry_mu;
std::set<const sdft_plan*> g_registry;

// process-wide schedule choice per log2 N for the FP32 path (autotuner)
std::atomic<int> g_choice[17];
// process-wide form of every length class for work-queue plans created later
std::atomic<int> g_rform[17];

int candidate_count(int logn, int dtype) {
    if (dtype != SDFT_F32) return split_kernel(logn, dtype) ? 1 : 0;
    int c = 0;
    while (f32_candidate(logn, c)) ++c;
    return c;
}

const KernelInfo* candidate(int logn, int dtype, int idx) {
    if (dtype != SDFT_F32) {
        const SplitInfo* si = split_kernel(logn, dtype);
        return (si && idx == 0) ? &si->kern : nullptr;
    }
    return f32_candidate(logn, idx);
}

bool plan_alive(const sdft_plan* p) {
    if (p == nullptr) return false;
    std::lock_guard<std::mutex> lk(g_registry_mu);
    return g_registry.count(p) != 0 && p->magic == kMagic;
}

int log2_exact(int64_t n) {
    if (n < 1) return -1;
    int m = 0;
    while (((int64_t)1 << m) < n) ++m;
    return (((int64_t)1 << m) == n) ? m : -1;
}

void free_plan_memory(sdft_plan* p) {
    if (p->d_tw) cudaFree(p->d_tw);
    if (p->d_scratch) cudaFree(p->d_scratch);
    if (p->d_status) cudaFree(p->d_status);
    if (p->d_aux) cudaFree(p->d_aux);
    for (int s = 0; s < 2; ++s) {
        for (int pl = 0; pl < 2; ++pl)
            if (p->host.d_buf[s][pl]) cudaFree(p->host.d_buf[s][pl]);
        if (p->host.streams[s]) cudaStreamDestroy(p->host.streams[s]);
    }
    if (p->host.start) cudaEventDestroy(p->host.start);
    if (p->host.d_scratch) cudaFree(p->host.d_scratch);
    RaggedState& r = p->rag;
    for (int d = 0; d < 2; ++d) {
        if (r.exec[d]) cudaGraphExecDestroy(r.exec[d]);
        if (r.graph[d]) cudaGraphDestroy(r.graph[d]);
    }
    if (r.d_offsets) cudaFree(r.d_offsets);
    for (int ph = 0; ph < kRaggedPhases; ++ph)
        if (r.d_items[ph]) cudaFree(r.d_items[ph]);
    if (r.d_sync) cudaFree(r.d_sync);
}

bool ranges_overlap(const void* a, const void* b, size_t bytes) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bytes && y < x + bytes;
}

int check_buffers(const sdft_plan* p, const float* xr, const float* xi, const float* yr,
                  const float* yi) {
    if (!xr || !xi || !yr || !yi) return SDFT_ERR_INVALID_ARG;
    const uintptr_t a[4] = {(uintptr_t)xr, (uintptr_t)xi, (uintptr_t)yr, (uintptr_t)yi};
    for (uintptr_t v : a)
        if (v % 16 != 0) return SDFT_ERR_MISALIGNED;
    const size_t bytes = (size_t)p->points * sizeof(float);
    // outputs must not overlap each other
    if (ranges_overlap(yr, yi, bytes)) return SDFT_ERR_ALIAS;
    // an output may coincide exactly with its own input (in place) and may
    // not otherwise overlap any input
    const bool in_place = (yr == xr) && (yi == xi);
    if (in_place) {
        if (ranges_overlap(yr, xi, bytes) || ranges_overlap(yi, xr, bytes)) return SDFT_ERR_ALIAS;
    } else {
        if (ranges_overlap(yr, xr, bytes) || ranges_overlap(yr, xi, bytes) ||
            ranges_overlap(yi, xr, bytes) || ranges_overlap(yi, xi, bytes))
            return SDFT_ERR_ALIAS;
    }
    return SDFT_OK;
}

int check_device(const sdft_plan* p) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SDFT_ERR_CUDA;
    return dev == p->device ? SDFT_OK : SDFT_ERR_INVALID_ARG;
}

int launch(const sdft_plan* p, int direction, const float* xr, const float* xi, float* yr,
           float* yi, cudaStream_t stream, long long batch, float2* scratch) {
    LaunchArgs a;
    a.xr = xr;
    a.xi = xi;
    a.yr = yr;
    a.yi = yi;
    a.batch = batch;
    a.tw = p->d_tw;
    a.w64 = p->w64;
    a.scratch = scratch;
    a.status = p->d_status;
    a.aux = p->d_aux;
    a.grid = p->grid;
    a.stream = stream;
    a.adj = (direction == SDFT_ADJOINT);
    // CTAs that have work: one per tile, or a whole cluster per transform
    const long long tiles = (batch + p->kern->transforms_per_cta - 1) /
                            p->kern->transforms_per_cta * std::max(1, p->kern->cluster);
    if (scratch == nullptr && tiles < a.grid) a.grid = (int)std::max<long long>(tiles, 1);
    return p->kern->launch(a) == cudaSuccess ? SDFT_OK : SDFT_ERR_CUDA;
}

// Ragged plans: launch the direction's graph, building it on first use and
// re-pointing its kernel node when its arguments change.
int launch_ragged(sdft_plan* p, int direction, const float* xr, const float* xi, float* yr,
                  float* yi, cudaStream_t stream) {
    RaggedState& r = p->rag;
    const int d = direction == SDFT_ADJOINT ? 1 : 0;
    RaggedArgs a = {};
    a.xr = xr;
    a.xi = xi;
    a.yr = yr;
    a.yi = yi;
    for (int ph = 0; ph < kRaggedPhases; ++ph) {
        a.items[ph] = r.d_items[ph];
        a.nitems[ph] = r.nitems[ph];
    }
    a.offsets = r.d_offsets;
    a.counters = r.d_sync;
    a.status = p->d_status;
    a.wait_polls = r.wait_polls;
    a.inject = r.inject;
    for (int c = 0; c < kRaggedRoutines; ++c) a.tw[c] = r.rtw[c];
    a.w = p->w64;
    void* kargs[] = {&a};
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void*>(ragged_kernel_fn(d == 1));
    kp.gridDim = dim3((unsigned)p->grid, 1, 1);
    kp.blockDim = dim3((unsigned)ragged_threads(), 1, 1);
    kp.sharedMemBytes = (unsigned)ragged_smem();
    kp.kernelParams = kargs;
    kp.extra = nullptr;
    std::lock_guard<std::mutex> lk(r.mu);
    if (!r.exec[d]) {
        if (cudaGraphCreate(&r.graph[d], 0) != cudaSuccess) return SDFT_ERR_CUDA;
        cudaMemsetParams mp = {};
        mp.dst = r.d_sync;
        mp.value = 0;
        mp.elementSize = sizeof(int);
        mp.width = kRaggedPhases + 1;
        mp.height = 1;
        mp.pitch = 0;
        cudaGraphNode_t mnode = nullptr;
        cudaKernelNodeAttrValue cl = {};
        cl.clusterDim.x = kRaggedCluster;
        cl.clusterDim.y = 1;
        cl.clusterDim.z = 1;
        if (cudaGraphAddMemsetNode(&mnode, r.graph[d], nullptr, 0, &mp) != cudaSuccess ||
            cudaGraphAddKernelNode(&r.knode[d], r.graph[d], &mnode, 1, &kp) != cudaSuccess ||
            cudaGraphKernelNodeSetAttribute(r.knode[d], cudaKernelNodeAttributeClusterDimension,
                                            &cl) != cudaSuccess ||
            cudaGraphInstantiate(&r.exec[d], r.graph[d], 0) != cudaSuccess) {
            if (r.graph[d]) cudaGraphDestroy(r.graph[d]);
            r.graph[d] = nullptr;
            r.exec[d] = nullptr;
            return SDFT_ERR_CUDA;
        }
        r.args[d] = a;
    } else if (std::memcmp(&r.args[d], &a, sizeof(a)) != 0) {
        if (cudaGraphExecKernelNodeSetParams(r.exec[d], r.knode[d], &kp) != cudaSuccess)
            return SDFT_ERR_CUDA;
        r.args[d] = a;
    }
    return cudaGraphLaunch(r.exec[d], stream) == cudaSuccess ? SDFT_OK : SDFT_ERR_CUDA;
}

// Device-side address of page-locked host memory the GPU can reach directly
// (null if `p` is not such memory).
const void* mapped_host(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();   // clear the error this query leaves for plain host memory
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost) ? a.devicePointer : nullptr;
}

int run(sdft_plan* p, int direction, const float* xr, const float* xi, float* yr, float* yi,
        cudaStream_t stream, long long batch, float2* scratch) {
    if (p->rag.on) return launch_ragged(p, direction, xr, xi, yr, yi, stream);
    return launch(p, direction, xr, xi, yr, yi, stream, batch, scratch);
}

// Work items of a work-queue plan (host only): for transforms of log2 lengths
// logn[] starting at start[] (floats) and the form of every length, one item
// per transform for the group phases (q = 8, 4, 2), longest first, and row
// tiles of `per_item` transforms for q = 1, longest first (ragged.h).
// `owner[t]` records (phase, item) of transform t.
struct RaggedWork {
    std::vector<int4> items[kRaggedPhases];
    std::vector<long long> order_off;            // row tiles: row starts in work order
    std::vector<std::pair<int, int>> owner;      // per transform: (phase, item)
};

int ragged_work(const signed char* logn, const long long* start, int64_t count,
                const int* form, RaggedWork& w) {
    unsigned classes = 0;
    for (int64_t t = 0; t < count; ++t) classes |= 1u << logn[t];
    w.owner.assign((size_t)count, std::make_pair(-1, -1));
    for (int l = kMaxLogN; l >= 2; --l) {
        if (!(classes & (1u << l))) continue;
        const RaggedForm* f = ragged_form(l, form[l]);
        if (!f) return SDFT_ERR_INVALID_ARG;
        const int ph = ragged_phase_of(f->q);
        if (f->q > 1) {
            for (int64_t t = 0; t < count; ++t)
                if (logn[t] == l) {
                    const long long o = start[t];
                    w.owner[(size_t)t] = std::make_pair(ph, (int)w.items[ph].size());
                    w.items[ph].push_back(make_int4(f->code, (int)(uint32_t)o,
                                                    (int)(uint32_t)((unsigned long long)o >> 32),
                                                    1 << l));
                }
        } else {
            const int first = (int)w.order_off.size();
            for (int64_t t = 0; t < count; ++t)
                if (logn[t] == l) {
                    w.owner[(size_t)t] = std::make_pair(
                        ph, (int)w.items[ph].size() + ((int)w.order_off.size() - first) / f->per_item);
                    w.order_off.push_back(start[t]);
                }
            const int n_in = (int)w.order_off.size() - first;
            for (int s0 = 0; s0 < n_in; s0 += f->per_item)
                w.items[ph].push_back(make_int4(f->code, first + s0, std::min(f->per_item, n_in - s0), 0));
        }
    }
    for (int ph = 0; ph < kRaggedPhases; ++ph)
        if ((int64_t)w.items[ph].size() > count) return SDFT_ERR_INVALID_ARG;
    return SDFT_OK;
}

// Upload a work-queue plan's items under its current forms on `st` (the
// caller synchronises).
int build_queue(sdft_plan* p, cudaStream_t st) {
    RaggedState& r = p->rag;
    RaggedWork w;
    try {
        const int s = ragged_work(r.logn.data(), r.start.data(), r.count, r.form, w);
        if (s != SDFT_OK) return s;
    } catch (...) {
        return SDFT_ERR_ALLOC;
    }
    for (int ph = 0; ph < kRaggedPhases; ++ph) {
        if (!w.items[ph].empty() &&
            cudaMemcpyAsync(r.d_items[ph], w.items[ph].data(), w.items[ph].size() * sizeof(int4),
                            cudaMemcpyHostToDevice, st) != cudaSuccess)
            return SDFT_ERR_CUDA;
        r.nitems[ph] = (int)w.items[ph].size();
    }
    if (!w.order_off.empty() &&
        cudaMemcpyAsync(r.d_offsets, w.order_off.data(), w.order_off.size() * sizeof(long long),
                        cudaMemcpyHostToDevice, st) != cudaSuccess)
        return SDFT_ERR_CUDA;
    return SDFT_OK;
}

// Rebuild a work-queue plan's items after a form change (synchronous; the
// plan must have no work in flight that reads its items).
int rebuild_queue(sdft_plan* p) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return SDFT_ERR_CUDA;
    int s = cudaDeviceSynchronize() == cudaSuccess ? SDFT_OK : SDFT_ERR_CUDA;
    if (s == SDFT_OK) s = build_queue(p, st);
    if (s == SDFT_OK && cudaStreamSynchronize(st) != cudaSuccess) s = SDFT_ERR_CUDA;
    cudaStreamDestroy(st);
    return s;
}

// Ragged plans, and uniform plans on the work-queue schedule: the persistent
// kernel of ragged.cu.  Every length class starts with the process-wide form
// selected for it; the twiddle tables of all forms of the plan's classes are
// made at creation, so that a form change only rebuilds the work items.
sdft_plan* create_queue_plan(const int64_t* lengths, int64_t count, bool uniform) {
    sdft_plan* p = new (std::nothrow) sdft_plan();
    if (!p) { fail(SDFT_ERR_ALLOC); return nullptr; }
    p->magic = 0;
    p->dtype = SDFT_F32;
    p->n = uniform ? lengths[0] : 0;
    p->batch = count;
    p->kern = nullptr;
    RaggedState& r = p->rag;
    r.on = true;
    r.uniform = uniform;
    r.count = count;
    int64_t total = 0;
    try {
        r.logn.resize((size_t)count);
        r.start.resize((size_t)count);
    } catch (...) {
        delete p;
        fail(SDFT_ERR_ALLOC);
        return nullptr;
    }
    for (int64_t t = 0; t < count; ++t) {
        const int l = log2_exact(lengths[t]);
        r.logn[(size_t)t] = (signed char)l;
        r.start[(size_t)t] = total;
        total += lengths[t];
        r.classes |= 1u << l;
    }
    p->points = total;
    for (int l = 2; l <= kMaxLogN; ++l) {
        const int f = g_rform[l].load();
        r.form[l] = (f >= 0 && f < ragged_form_count(l)) ? f : 0;
    }
    int status = SDFT_OK;
    cudaStream_t st = nullptr;
    do {
        if (cudaGetDevice(&p->device) != cudaSuccess) { status = SDFT_ERR_CUDA; break; }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
            status = SDFT_ERR_CUDA; break;
        }
        if (ragged_prepare() != cudaSuccess) { status = SDFT_ERR_CUDA; break; }
        p->grid = ragged_resident_ctas();
        if (p->grid < kRaggedCluster) { status = SDFT_ERR_CUDA; break; }
        p->occupancy = (p->grid + sms - 1) / sms;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            status = SDFT_ERR_CUDA; break;
        }
        // twiddle tables of every form of every class present
        int64_t tw_total = 64;
        int64_t base[kRaggedRoutines] = {};
        for (int l = 2; l <= kMaxLogN; ++l) {
            if (!(r.classes & (1u << l))) continue;
            for (int f = 0; f < ragged_form_count(l); ++f) {
                const RaggedForm* fm = ragged_form(l, f);
                base[fm->code] = tw_total;
                tw_total += std::max<int64_t>(fm->tw_entries, 1);
            }
        }
        const size_t cap = (size_t)std::max<int64_t>(count, 1);
        bool ok = cudaMalloc(&p->d_tw, tw_total * sizeof(float2)) == cudaSuccess &&
                  cudaMalloc(&p->d_status, sizeof(int)) == cudaSuccess &&
                  cudaMalloc(&r.d_sync, (kRaggedPhases + 1) * sizeof(int)) == cudaSuccess &&
                  cudaMalloc(&r.d_offsets, cap * sizeof(long long)) == cudaSuccess;
        for (int ph = 0; ph < kRaggedPhases && ok; ++ph)
            ok = cudaMalloc(&r.d_items[ph], cap * sizeof(int4)) == cudaSuccess;
        if (!ok) { status = SDFT_ERR_ALLOC; break; }
        if (cudaMemsetAsync(p->d_status, 0, sizeof(int), st) != cudaSuccess ||
            cudaMemsetAsync(r.d_sync, 0, (kRaggedPhases + 1) * sizeof(int), st) != cudaSuccess) {
            status = SDFT_ERR_CUDA; break;
        }
        if (make_w64(&p->w64, p->d_tw, st) != cudaSuccess) { status = SDFT_ERR_CUDA; break; }
        for (int l = 2; l <= kMaxLogN && status == SDFT_OK; ++l) {
            if (!(r.classes & (1u << l))) continue;
            for (int f = 0; f < ragged_form_count(l) && status == SDFT_OK; ++f) {
                const RaggedForm* fm = ragged_form(l, f);
                r.rtw[fm->code] = p->d_tw + base[fm->code];
                if (fm->ntables > 0 &&
                    make_tables(p->d_tw + base[fm->code], fm->tables, fm->ntables, st) != cudaSuccess)
                    status = SDFT_ERR_CUDA;
            }
        }
        if (status != SDFT_OK) break;
        status = build_queue(p, st);
        if (status != SDFT_OK) break;
        if (cudaStreamSynchronize(st) != cudaSuccess) { status = SDFT_ERR_CUDA; break; }
    } while (0);
    if (st) cudaStreamDestroy(st);
    if (status != SDFT_OK) {
        free_plan_memory(p);
        delete p;
        fail(status);
        return nullptr;
    }
    p->magic = kMagic;
    {
        std::lock_guard<std::mutex> lk(g_registry_mu);
        g_registry.insert(p);
    }
    return p;
}

}  // namespace

extern "C" {

const char* sdft_version(void) { return "0.1.0"; }

int sdft_last_error(void) { return g_last_error; }

const char* sdft_status_string(int status) {
    switch (status) {
        case SDFT_OK: return "ok";
        case SDFT_ERR_INVALID_ARG: return "invalid argument";
        case SDFT_ERR_UNSUPPORTED_N: return "unsupported transform length (need a power of two in [2, 65536])";
        case SDFT_ERR_MISALIGNED: return "data pointer not 16-byte aligned";
        case SDFT_ERR_ALIAS: return "input and output arrays partially overlap";
        case SDFT_ERR_BAD_PLAN: return "invalid or destroyed plan";
        case SDFT_ERR_CUDA: return "CUDA runtime error";
        case SDFT_ERR_ALLOC: return "allocation failed";
        case SDFT_ERR_TIMEOUT: return "bounded device wait timed out";
        case SDFT_ERR_UNSUPPORTED_DTYPE: return "unsupported dtype";
        default: return "unknown status";
    }
}

sdft_plan* plan_create_idx(int64_t n, int64_t batch, int dtype, int idx);

sdft_plan* sdft_plan_create(int64_t n, int64_t batch, int dtype) {
    NvtxRange range("sdft_plan_create");
    const int logn = log2_exact(n);
    const int idx = (logn >= 1 && logn <= kMaxLogN && dtype == SDFT_F32) ? g_choice[logn].load() : 0;
    return plan_create_idx(n, batch, dtype, idx);
}

sdft_plan* plan_create_idx(int64_t n, int64_t batch, int dtype, int idx) {
    const int logn = log2_exact(n);
    if (logn < 1 || logn > kMaxLogN) { fail(SDFT_ERR_UNSUPPORTED_N); return nullptr; }
    if (batch < 1) { fail(SDFT_ERR_INVALID_ARG); return nullptr; }
    if (dtype != SDFT_F32 && dtype != SDFT_F32_SPLIT_BF16 && dtype != SDFT_F32_SPLIT_FP16) {
        fail(SDFT_ERR_UNSUPPORTED_DTYPE);
        return nullptr;
    }
    if (batch > ((int64_t)1 << 40) / n) { fail(SDFT_ERR_INVALID_ARG); return nullptr; }

    const SplitInfo* si = nullptr;
    const KernelInfo* k = nullptr;
    if (dtype == SDFT_F32) {
        k = f32_candidate(logn, idx);
        if (!k) k = f32_candidate(logn, 0);
    } else {
        si = split_kernel(logn, dtype);   // tensor-core path: N = 256 and 1024
        if (!si) { fail(SDFT_ERR_UNSUPPORTED_DTYPE); return nullptr; }
        k = &si->kern;
    }
    if (!k) { fail(SDFT_ERR_UNSUPPORTED_N); return nullptr; }
    if (k->queue) {
        std::vector<int64_t> lengths((size_t)batch, n);
        return create_queue_plan(lengths.data(), batch, true);
    }

    sdft_plan* p = new (std::nothrow) sdft_plan();
    if (!p) { fail(SDFT_ERR_ALLOC); return nullptr; }
    p->magic = 0;
    p->dtype = dtype;
    p->n = n;
    p->batch = batch;
    p->points = n * batch;
    p->kern = k;
    int status = SDFT_OK;
    cudaStream_t st = nullptr;
    do {
        if (cudaGetDevice(&p->device) != cudaSuccess) { status = SDFT_ERR_CUDA; break; }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
            status = SDFT_ERR_CUDA; break;
        }
        if (k->prepare() != cudaSuccess) { status = SDFT_ERR_CUDA; break; }
        p->occupancy = k->blocks_per_sm();
        const int bps = std::max(1, p->occupancy);
        p->grid = bps * sms;
        if (k->resident_ctas) {              // cluster kernels: whole clusters only
            p->grid = k->resident_ctas();
            if (p->grid < std::max(1, k->cluster)) { status = SDFT_ERR_CUDA; break; }
        }
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            status = SDFT_ERR_CUDA; break;
        }
        const int64_t tw_entries = std::max<int64_t>(k->tw_entries, 64);
        if (cudaMalloc(&p->d_tw, tw_entries * sizeof(float2)) != cudaSuccess) {
            status = SDFT_ERR_ALLOC; break;
        }
        if (cudaMalloc(&p->d_status, sizeof(int)) != cudaSuccess) { status = SDFT_ERR_ALLOC; break; }
        if (cudaMemsetAsync(p->d_status, 0, sizeof(int), st) != cudaSuccess) { status = SDFT_ERR_CUDA; break; }
        if (k->scratch_per_cta > 0) {
            const size_t bytes = (size_t)p->grid * (size_t)k->scratch_per_cta * sizeof(float2);
            if (cudaMalloc(&p->d_scratch, bytes) != cudaSuccess) { status = SDFT_ERR_ALLOC; break; }
        }
        // the register constants first (uses the table memory as scratch)
        if (make_w64(&p->w64, p->d_tw, st) != cudaSuccess) { status = SDFT_ERR_CUDA; break; }
        if (make_tables(p->d_tw, k->tables, k->ntables, st) != cudaSuccess) { status = SDFT_ERR_CUDA; break; }
        if (si) {
            if (cudaMalloc(&p->d_aux, si->aux_bytes) != cudaSuccess) { status = SDFT_ERR_ALLOC; break; }
            if (si->make_aux(p->d_aux, st) != cudaSuccess) { status = SDFT_ERR_CUDA; break; }
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) { status = SDFT_ERR_CUDA; break; }
    } while (0);
    if (st) cudaStreamDestroy(st);
    if (status != SDFT_OK) {
        free_plan_memory(p);
        delete p;
        fail(status);
        return nullptr;
    }
    p->magic = kMagic;
    {
        std::lock_guard<std::mutex> lk(g_registry_mu);
        g_registry.insert(p);
    }
    return p;
}

sdft_plan* sdft_plan_create_ragged(const int64_t* lengths, int64_t count, int dtype) {
    NvtxRange range("sdft_plan_create_ragged");
    if (lengths == nullptr || count < 1 || count > ((int64_t)1 << 31)) {
        fail(SDFT_ERR_INVALID_ARG);
        return nullptr;
    }
    if (dtype != SDFT_F32 && dtype != SDFT_F32_SPLIT_BF16 && dtype != SDFT_F32_SPLIT_FP16) {
        fail(SDFT_ERR_UNSUPPORTED_DTYPE);
        return nullptr;
    }
    int64_t total = 0;
    for (int64_t t = 0; t < count; ++t) {
        const int l = log2_exact(lengths[t]);
        if (l < 2 || l > kMaxLogN) { fail(SDFT_ERR_UNSUPPORTED_N); return nullptr; }
        total += lengths[t];
        if (total > ((int64_t)1 << 40)) { fail(SDFT_ERR_INVALID_ARG); return nullptr; }
    }
    if (dtype != SDFT_F32) { fail(SDFT_ERR_UNSUPPORTED_DTYPE); return nullptr; }
    return create_queue_plan(lengths, count, false);
}

void sdft_plan_destroy(sdft_plan* plan) {
    if (plan == nullptr) return;
    {
        std::lock_guard<std::mutex> lk(g_registry_mu);
        if (g_registry.erase(plan) == 0) return;  // not ours, or already destroyed
    }
    plan->magic = 0;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != plan->device) cudaSetDevice(plan->device);
    free_plan_memory(plan);
    if (cur >= 0 && cur != plan->device) cudaSetDevice(cur);
    delete plan;
}

int sdft_execute(const sdft_plan* plan, int direction, const float* xr, const float* xi,
                 float* yr, float* yi, void* stream) {
    NvtxRange range(direction == SDFT_ADJOINT ? "sdft_adjoint" : "sdft_forward");
    if (!plan_alive(plan)) return fail(SDFT_ERR_BAD_PLAN);
    if (direction != SDFT_FORWARD && direction != SDFT_ADJOINT) return fail(SDFT_ERR_INVALID_ARG);
    int s = check_buffers(plan, xr, xi, yr, yi);
    if (s != SDFT_OK) return fail(s);
    s = check_device(plan);
    if (s != SDFT_OK) return fail(s);
    s = run(const_cast<sdft_plan*>(plan), direction, xr, xi, yr, yi, (cudaStream_t)stream,
            plan->batch, plan->d_scratch);
    if (s != SDFT_OK) return fail(s);
    return SDFT_OK;
}

int sdft_forward(const sdft_plan* plan, const float* xr, const float* xi, float* yr, float* yi,
                 void* stream) {
    return sdft_execute(plan, SDFT_FORWARD, xr, xi, yr, yi, stream);
}

int sdft_adjoint(const sdft_plan* plan, const float* xr, const float* xi, float* yr, float* yi,
                 void* stream) {
    return sdft_execute(plan, SDFT_ADJOINT, xr, xi, yr, yi, stream);
}

int sdft_execute_host(sdft_plan* plan, int direction, const float* xr, const float* xi, float* yr,
                      float* yi, void* stream) {
    NvtxRange range("sdft_execute_host");
    if (!plan_alive(plan)) return fail(SDFT_ERR_BAD_PLAN);
    if (direction != SDFT_FORWARD && direction != SDFT_ADJOINT) return fail(SDFT_ERR_INVALID_ARG);
    if (!xr || !xi || !yr || !yi) return fail(SDFT_ERR_INVALID_ARG);
    int s = check_device(plan);
    if (s != SDFT_OK) return fail(s);
    HostStaging& h = plan->host;
    const int64_t n = plan->n;
    const bool rag = plan->rag.on;
    if (h.mode != SDFT_HOST_STAGED) {
        // zero copy: the kernel reads and writes the page-locked host buffers
        // directly over the CPU-GPU link (no staging, no copy engines)
        const float* dxr = static_cast<const float*>(mapped_host(xr));
        const float* dxi = static_cast<const float*>(mapped_host(xi));
        float* dyr = static_cast<float*>(const_cast<void*>(mapped_host(yr)));
        float* dyi = static_cast<float*>(const_cast<void*>(mapped_host(yi)));
        if (dxr && dxi && dyr && dyi) {
            s = check_buffers(plan, dxr, dxi, dyr, dyi);
            if (s != SDFT_OK) return fail(s);
            cudaStream_t user = (cudaStream_t)stream;
            s = run(plan, direction, dxr, dxi, dyr, dyi, user, plan->batch, plan->d_scratch);
            if (s != SDFT_OK) return fail(s);
            return cudaStreamSynchronize(user) == cudaSuccess ? SDFT_OK : fail(SDFT_ERR_CUDA);
        }
        if (h.mode == SDFT_HOST_ZERO_COPY) return fail(SDFT_ERR_INVALID_ARG);
    }
    if (h.chunk == 0) {
        // ~32 MiB per plane per slot, whole transforms, at least one; a ragged
        // plan moves its whole batch as one chunk
        int64_t chunk = rag ? plan->batch
                            : std::max<int64_t>(1, ((int64_t)32 << 20) / (n * (int64_t)sizeof(float)));
        chunk = std::min<int64_t>(chunk, plan->batch);
        const int64_t chunk_points = rag ? plan->points : chunk * n;
        // Each resource is created only if an earlier, failed set-up has not
        // already made it, so a retry completes the set-up instead of leaking
        // (the sizes depend on the plan alone); the plan frees them all.
        for (int sl = 0; sl < 2; ++sl) {
            for (int pl = 0; pl < 2; ++pl)
                if (!h.d_buf[sl][pl] &&
                    cudaMalloc(&h.d_buf[sl][pl], (size_t)chunk_points * sizeof(float)) != cudaSuccess) {
                    h.d_buf[sl][pl] = nullptr;
                    return fail(SDFT_ERR_ALLOC);
                }
            if (!h.streams[sl] &&
                cudaStreamCreateWithFlags(&h.streams[sl], cudaStreamNonBlocking) != cudaSuccess) {
                h.streams[sl] = nullptr;
                return fail(SDFT_ERR_CUDA);
            }
        }
        if (!h.start && cudaEventCreateWithFlags(&h.start, cudaEventDisableTiming) != cudaSuccess) {
            h.start = nullptr;
            return fail(SDFT_ERR_CUDA);
        }
        // a work-queue plan moves its batch as one chunk (slot 0 only)
        const int64_t scr = rag ? 0 : plan->kern->scratch_per_cta;
        if (scr > 0 && !h.d_scratch) {
            const size_t sb = (size_t)plan->grid * (size_t)scr * sizeof(float2);
            if (cudaMalloc(&h.d_scratch, sb) != cudaSuccess) {
                h.d_scratch = nullptr;
                return fail(SDFT_ERR_ALLOC);
            }
        }
        h.chunk = chunk;
    }
    cudaStream_t user = (cudaStream_t)stream;
    if (cudaEventRecord(h.start, user) != cudaSuccess) return fail(SDFT_ERR_CUDA);
    for (int sl = 0; sl < 2; ++sl)
        if (cudaStreamWaitEvent(h.streams[sl], h.start, 0) != cudaSuccess) return fail(SDFT_ERR_CUDA);
    const int64_t nchunks = (plan->batch + h.chunk - 1) / h.chunk;
    for (int64_t c = 0; c < nchunks; ++c) {
        const int sl = (int)(c & 1);
        cudaStream_t st = h.streams[sl];
        const int64_t b0 = c * h.chunk;
        const int64_t nb = std::min<int64_t>(h.chunk, plan->batch - b0);
        const size_t off = rag ? 0 : (size_t)b0 * n;
        const size_t bytes = (rag ? (size_t)plan->points : (size_t)nb * n) * sizeof(float);
        float* dr = h.d_buf[sl][0];
        float* di = h.d_buf[sl][1];
        if (cudaMemcpyAsync(dr, xr + off, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(di, xi + off, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return fail(SDFT_ERR_CUDA);
        s = run(plan, direction, dr, di, dr, di, st, nb, sl == 0 ? plan->d_scratch : h.d_scratch);
        if (s != SDFT_OK) return fail(s);
        if (cudaMemcpyAsync(yr + off, dr, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(yi + off, di, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return fail(SDFT_ERR_CUDA);
    }
    for (int sl = 0; sl < 2; ++sl)
        if (cudaStreamSynchronize(h.streams[sl]) != cudaSuccess) return fail(SDFT_ERR_CUDA);
    return SDFT_OK;
}

int sdft_plan_set_grid(sdft_plan* plan, int grid) {
    if (!plan_alive(plan)) return fail(SDFT_ERR_BAD_PLAN);
    if (grid < 1 || grid > (1 << 20)) return fail(SDFT_ERR_INVALID_ARG);
    // kernels with per-CTA scratch own exactly `grid` slots; their grid is fixed
    if (plan->d_scratch || plan->rag.on) return fail(SDFT_ERR_INVALID_ARG);
    plan->grid = grid;
    return SDFT_OK;
}

int sdft_plan_grid(const sdft_plan* plan) { return plan_alive(plan) ? plan->grid : 0; }

int sdft_plan_set_wait_limit(sdft_plan* plan, int polls) {
    if (!plan_alive(plan)) return fail(SDFT_ERR_BAD_PLAN);
    if (!plan->rag.on || polls < 1) return fail(SDFT_ERR_INVALID_ARG);
    plan->rag.wait_polls = polls;
    return SDFT_OK;
}

int sdft_plan_inject_unreachable_wait(sdft_plan* plan, int on) {
    if (!plan_alive(plan)) return fail(SDFT_ERR_BAD_PLAN);
    if (!plan->rag.on || plan->rag.nitems[0] + plan->rag.nitems[1] + plan->rag.nitems[2] == 0)
        return fail(SDFT_ERR_INVALID_ARG);
    plan->rag.inject = on ? 1 : 0;
    return SDFT_OK;
}

int sdft_plan_set_host_mode(sdft_plan* plan, int mode) {
    if (!plan_alive(plan)) return fail(SDFT_ERR_BAD_PLAN);
    if (mode != SDFT_HOST_AUTO && mode != SDFT_HOST_STAGED && mode != SDFT_HOST_ZERO_COPY)
        return fail(SDFT_ERR_INVALID_ARG);
    plan->host.mode = mode;
    return SDFT_OK;
}

int sdft_plan_sync_status(const sdft_plan* plan, void* stream) {
    if (!plan_alive(plan)) return fail(SDFT_ERR_BAD_PLAN);
    int s = check_device(plan);
    if (s != SDFT_OK) return fail(s);
    int h = 0;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemcpyAsync(&h, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemsetAsync(plan->d_status, 0, sizeof(int), st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return fail(SDFT_ERR_CUDA);
    return h == 0 ? SDFT_OK : fail(h);
}

int64_t sdft_plan_n(const sdft_plan* plan) { return plan_alive(plan) ? plan->n : 0; }
int64_t sdft_plan_batch(const sdft_plan* plan) { return plan_alive(plan) ? plan->batch : 0; }
int64_t sdft_plan_points(const sdft_plan* plan) { return plan_alive(plan) ? plan->points : 0; }
int sdft_plan_dtype(const sdft_plan* plan) { return plan_alive(plan) ? plan->dtype : -1; }

int sdft_plan_launches(const sdft_plan* plan, int direction) {
    (void)direction;
    if (!plan_alive(plan)) return 0;
    return plan->rag.on ? 1 : plan->kern->launches;
}

int sdft_plan_describe(const sdft_plan* plan, char* buf, int64_t len) {
    if (!plan_alive(plan)) return fail(SDFT_ERR_BAD_PLAN), -1;
    if (plan->rag.on) {
        const RaggedState& r = plan->rag;
        char cls[512] = {0};
        int o = 0;
        for (int l = 2; l <= kMaxLogN && o < (int)sizeof(cls); ++l)
            if (r.classes & (1u << l)) {
                const RaggedForm* f = ragged_form(l, r.form[l]);
                o += std::snprintf(cls + o, sizeof(cls) - (size_t)o, "%s%d: form %d (%s)",
                                   o ? "; " : "", 1 << l, r.form[l],
                                   f->q > 1 ? (f->q == 8 ? "8 CTAs" : f->q == 4 ? "4 CTAs" : "2 CTAs")
                                            : "row tile");
            }
        const char* head = r.uniform ? (queue_candidate(log2_exact(plan->n))
                                            ? queue_candidate(log2_exact(plan->n))->name
                                            : "work queue")
                                     : "ragged";
        return std::snprintf(buf, buf ? (size_t)std::max<int64_t>(len, 0) : 0,
                             "%s: %lld transforms, %lld points, {%s}; one persistent launch "
                             "(graph: counter memset + kernel), %d threads/CTA, %zu B smem, "
                             "clusters of %d, grid %d, items per phase (8/4/2 CTAs, rows) "
                             "%d/%d/%d/%d",
                             head, (long long)r.count, (long long)plan->points, cls,
                             ragged_threads(), ragged_smem(), kRaggedCluster, plan->grid,
                             r.nitems[0], r.nitems[1], r.nitems[2], r.nitems[3]);
    }
    return std::snprintf(buf, buf ? (size_t)std::max<int64_t>(len, 0) : 0,
                         "%s; %d threads/CTA, %zu B smem, grid %d (occupancy %d), "
                         "%d transform(s)/CTA tile",
                         plan->kern->name, plan->kern->threads, plan->kern->smem, plan->grid,
                         plan->occupancy, plan->kern->transforms_per_cta);
}

int sdft_schedule_count(int64_t n, int dtype) {
    const int logn = log2_exact(n);
    if (logn < 1 || logn > kMaxLogN) return -fail(SDFT_ERR_UNSUPPORTED_N);
    const int c = candidate_count(logn, dtype);
    return c > 0 ? c : -fail(SDFT_ERR_UNSUPPORTED_DTYPE);
}

int sdft_schedule_describe(int64_t n, int dtype, int index, char* buf, int64_t len) {
    const int logn = log2_exact(n);
    if (logn < 1 || logn > kMaxLogN) return -fail(SDFT_ERR_UNSUPPORTED_N);
    const KernelInfo* k = candidate(logn, dtype, index);
    if (!k) return -fail(SDFT_ERR_INVALID_ARG);
    if (k->queue)
        return std::snprintf(buf, buf ? (size_t)std::max<int64_t>(len, 0) : 0,
                             "%s; %d threads/CTA, %zu B smem, persistent", k->name,
                             ragged_threads(), ragged_smem());
    return std::snprintf(buf, buf ? (size_t)std::max<int64_t>(len, 0) : 0,
                         "%s; %d threads/CTA, %zu B smem, %d transform(s)/CTA tile", k->name,
                         k->threads, k->smem, k->transforms_per_cta);
}

int sdft_schedule_select(int64_t n, int dtype, int index) {
    const int logn = log2_exact(n);
    if (logn < 1 || logn > kMaxLogN) return fail(SDFT_ERR_UNSUPPORTED_N);
    if (!candidate(logn, dtype, index)) return fail(SDFT_ERR_INVALID_ARG);
    if (dtype == SDFT_F32) g_choice[logn].store(index);
    return SDFT_OK;
}

int sdft_schedule_selected(int64_t n, int dtype) {
    const int logn = log2_exact(n);
    if (logn < 1 || logn > kMaxLogN) return -fail(SDFT_ERR_UNSUPPORTED_N);
    if (candidate_count(logn, dtype) == 0) return -fail(SDFT_ERR_UNSUPPORTED_DTYPE);
    return dtype == SDFT_F32 ? g_choice[logn].load() : 0;
}

int sdft_ragged_form_count(int64_t n) {
    const int l = log2_exact(n);
    const int c = (l >= 2 && l <= kMaxLogN) ? ragged_form_count(l) : 0;
    return c > 0 ? c : -fail(SDFT_ERR_UNSUPPORTED_N);
}

int sdft_ragged_form_describe(int64_t n, int form, char* buf, int64_t len) {
    const int l = log2_exact(n);
    const RaggedForm* f = (l >= 2 && l <= kMaxLogN) ? ragged_form(l, form) : nullptr;
    if (!f) return -fail(l >= 2 && l <= kMaxLogN ? SDFT_ERR_INVALID_ARG : SDFT_ERR_UNSUPPORTED_N);
    return std::snprintf(buf, buf ? (size_t)std::max<int64_t>(len, 0) : 0, "%s", f->name);
}

int sdft_ragged_form_select(int64_t n, int form) {
    const int l = log2_exact(n);
    if (l < 2 || l > kMaxLogN) return fail(SDFT_ERR_UNSUPPORTED_N);
    if (!ragged_form(l, form)) return fail(SDFT_ERR_INVALID_ARG);
    g_rform[l].store(form);
    return SDFT_OK;
}

int sdft_ragged_form_selected(int64_t n) {
    const int l = log2_exact(n);
    if (l < 2 || l > kMaxLogN) return -fail(SDFT_ERR_UNSUPPORTED_N);
    return g_rform[l].load();
}

int sdft_plan_set_ragged_form(sdft_plan* plan, int64_t n, int form) {
    if (!plan_alive(plan)) return fail(SDFT_ERR_BAD_PLAN);
    const int l = log2_exact(n);
    if (!plan->rag.on || l < 2 || l > kMaxLogN || !(plan->rag.classes & (1u << l)) ||
        !ragged_form(l, form))
        return fail(SDFT_ERR_INVALID_ARG);
    int s = check_device(plan);
    if (s != SDFT_OK) return fail(s);
    RaggedState& r = plan->rag;
    if (r.form[l] == form) return SDFT_OK;
    const int prev = r.form[l];
    r.form[l] = form;
    s = rebuild_queue(plan);
    if (s != SDFT_OK) {
        r.form[l] = prev;
        rebuild_queue(plan);
        return fail(s);
    }
    return SDFT_OK;
}

int sdft_ragged_work_layout(const int64_t* lengths, int64_t count, int32_t* phase_of,
                            int32_t* item_of, int64_t* nitems) {
    if (lengths == nullptr || count < 1 || count > ((int64_t)1 << 31) || !phase_of || !item_of ||
        !nitems)
        return fail(SDFT_ERR_INVALID_ARG);
    try {
        std::vector<signed char> logn((size_t)count);
        std::vector<long long> start((size_t)count);
        long long total = 0;
        for (int64_t t = 0; t < count; ++t) {
            const int l = log2_exact(lengths[t]);
            if (l < 2 || l > kMaxLogN) return fail(SDFT_ERR_UNSUPPORTED_N);
            logn[(size_t)t] = (signed char)l;
            start[(size_t)t] = total;
            total += lengths[t];
        }
        int form[17] = {};
        for (int l = 2; l <= kMaxLogN; ++l) form[l] = g_rform[l].load();
        RaggedWork w;
        const int s = ragged_work(logn.data(), start.data(), count, form, w);
        if (s != SDFT_OK) return fail(s);
        for (int64_t t = 0; t < count; ++t) {
            phase_of[t] = w.owner[(size_t)t].first;
            item_of[t] = w.owner[(size_t)t].second;
        }
        for (int ph = 0; ph < kRaggedPhases; ++ph) nitems[ph] = (int64_t)w.items[ph].size();
    } catch (...) {
        return fail(SDFT_ERR_ALLOC);
    }
    return SDFT_OK;
}

int sdft_plan_ragged_form(const sdft_plan* plan, int64_t n) {
    if (!plan_alive(plan)) return -fail(SDFT_ERR_BAD_PLAN);
    const int l = log2_exact(n);
    if (!plan->rag.on || l < 2 || l > kMaxLogN || !(plan->rag.classes & (1u << l)))
        return -fail(SDFT_ERR_INVALID_ARG);
    return plan->rag.form[l];
}

int sdft_plan_ragged_autotune(sdft_plan* plan, const float* xr, const float* xi, float* yr,
                              float* yi, int reps, void* stream) {
    NvtxRange range("sdft_plan_ragged_autotune");
    if (!plan_alive(plan)) return -fail(SDFT_ERR_BAD_PLAN);
    if (!plan->rag.on || reps < 1) return -fail(SDFT_ERR_INVALID_ARG);
    int s = check_device(plan);
    if (s == SDFT_OK) s = check_buffers(plan, xr, xi, yr, yi);
    if (s != SDFT_OK) return -fail(s);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return -fail(SDFT_ERR_CUDA);
    }
    RaggedState& r = plan->rag;
    // milliseconds per forward call with the current forms (one untimed call first)
    auto time_plan = [&](float& ms) {
        int q = run(plan, SDFT_FORWARD, xr, xi, yr, yi, st, plan->batch, nullptr);
        if (q == SDFT_OK && cudaEventRecord(e0, st) != cudaSuccess) q = SDFT_ERR_CUDA;
        for (int i = 0; i < reps && q == SDFT_OK; ++i)
            q = run(plan, SDFT_FORWARD, xr, xi, yr, yi, st, plan->batch, nullptr);
        if (q == SDFT_OK && (cudaEventRecord(e1, st) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            q = SDFT_ERR_CUDA;
        ms /= (float)reps;
        return q;
    };
    // greedy, one length class at a time, longest first: each form of the
    // class in turn, keeping another form only if it is faster by more than 1 %
    float best = 0.f;
    s = time_plan(best);
    for (int l = kMaxLogN; l >= 2 && s == SDFT_OK; --l) {
        if (!(r.classes & (1u << l)) || ragged_form_count(l) < 2) continue;
        const int keep0 = r.form[l];
        int keep = keep0;
        for (int f = 0; f < ragged_form_count(l) && s == SDFT_OK; ++f) {
            if (f == keep0) continue;
            r.form[l] = f;
            s = rebuild_queue(plan);
            float ms = 0.f;
            if (s == SDFT_OK) s = time_plan(ms);
            if (s == SDFT_OK && ms < best * 0.99f) { keep = f; best = ms; }
        }
        r.form[l] = keep;
        const int q = rebuild_queue(plan);
        if (s == SDFT_OK) s = q;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != SDFT_OK) return -fail(s);
    int mask = 0;
    for (int l = 2; l <= kMaxLogN; ++l)
        if ((r.classes & (1u << l)) && r.form[l] != 0) mask |= 1 << l;
    return mask;
}

int sdft_autotune(int64_t n, int64_t batch, int dtype, const float* xr, const float* xi, float* yr,
                  float* yi, int reps, float* ms_out, void* stream) {
    NvtxRange range("sdft_autotune");
    const int logn = log2_exact(n);
    if (logn < 1 || logn > kMaxLogN) return -fail(SDFT_ERR_UNSUPPORTED_N);
    if (batch < 1 || reps < 1) return -fail(SDFT_ERR_INVALID_ARG);
    const int count = candidate_count(logn, dtype);
    if (count == 0) return -fail(SDFT_ERR_UNSUPPORTED_DTYPE);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return -fail(SDFT_ERR_CUDA);
    }
    int best = -1;
    float best_ms = 0.f;
    int status = SDFT_OK;
    for (int idx = 0; idx < count && status == SDFT_OK; ++idx) {
        sdft_plan* p = plan_create_idx(n, batch, dtype, idx);
        if (!p) { status = g_last_error; break; }
        float ms = 0.f;
        int s = check_buffers(p, xr, xi, yr, yi);
        for (int w = 0; w < 2 && s == SDFT_OK; ++w)
            s = run(p, SDFT_FORWARD, xr, xi, yr, yi, st, batch, p->d_scratch);
        if (s == SDFT_OK && cudaEventRecord(e0, st) != cudaSuccess) s = SDFT_ERR_CUDA;
        for (int r = 0; r < reps && s == SDFT_OK; ++r)
            s = run(p, SDFT_FORWARD, xr, xi, yr, yi, st, batch, p->d_scratch);
        if (s == SDFT_OK && (cudaEventRecord(e1, st) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            s = SDFT_ERR_CUDA;
        sdft_plan_destroy(p);
        if (s != SDFT_OK) { status = s; break; }
        ms /= (float)reps;
        if (ms_out) ms_out[idx] = ms;
        if (best < 0 || ms < best_ms) { best = idx; best_ms = ms; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != SDFT_OK) return -fail(status);
    if (dtype == SDFT_F32) g_choice[logn].store(best);
    return best;
}

}  // extern "C"
