// noalloc.cu -- an allocation-free entry point for the long-transform kernel.
//
// The long-transform kernel (N = 32768 and 65536, kernels_large.cu) needs
// global scratch memory: each CTA runs its transform as two passes through a
// private N-point slot.  sdft_plan_create allocates that scratch (and the
// twiddle tables) with cudaMalloc.  Some callers cannot do that: code whose
// device memory is entirely owned by another allocator (a framework's caching
// pool, a fixed arena sized at start-up), code running under a per-process
// memory cap, or latency-critical code that must not risk the device-wide
// synchronisation cudaMalloc and cudaFree can cause.  sdft_execute_noalloc
// serves them: it runs the same kernel on scratch and tables that live in
// file-scope __device__ arrays, loaded with the library and held by every
// GPU that loads it until the process exits.  It calls no cudaMalloc,
// cudaFree or other allocating routine.
//
// Limits and sharing:
//   * scratch: kNoAllocScratch float2 entries (8 MiB), i.e. 16 transform slots
//     of N = 65536 or 32 of N = 32768; a call uses min(batch, slots) CTAs and
//     any batch size is processed by those CTAs in turn.
//   * Every call shares the arrays.  Calls that overlap on the GPU (two
//     streams, or two host threads) race on the scratch and corrupt each
//     other's results; order them on one stream.
//   * The scratch keeps the last call's contents; nothing in it needs to start
//     at zero, because every slot is fully written before it is read.
//   * The first call on each device does a one-time set-up with that device
//     current: it resolves the arrays' device addresses, sets the kernel's
//     shared-memory limit, fills the twiddle tables and synchronises the
//     device.  Make that first call before any stream capture.
// The paper has no counterpart to this entry point.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/sdft.h"
#include "launch.h"

namespace sdft {
namespace {

constexpr int64_t kNoAllocScratch = (int64_t)16 * 65536;            // float2 entries, 8 MiB
constexpr int64_t kTw15 = 256 + 128 + 32768;                         // tables of N = 32768
constexpr int64_t kTw16 = 256 + 256 + 65536;                         // tables of N = 65536
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float2 g_noalloc_scratch[kNoAllocScratch];
static __device__ __align__(256) float2 g_noalloc_tables[kTw15 + kTw16];
static __device__ __align__(256) float2 g_noalloc_w64[64];

struct DeviceState {
    bool ready = false;
    float2* scratch = nullptr;   // device address of g_noalloc_scratch
    float2* tables = nullptr;    // device address of g_noalloc_tables
    W64 w64 = {};
};

std::mutex g_mu;
DeviceState g_state[kMaxDevices];

// One-time per-device set-up (the device is current).  Synchronises.
int setup(int dev) {
    DeviceState& s = g_state[dev];
    if (s.ready) return SDFT_OK;
    void* scratch = nullptr;
    void* tables = nullptr;
    void* w64 = nullptr;
    if (cudaGetSymbolAddress(&scratch, g_noalloc_scratch) != cudaSuccess) return SDFT_ERR_CUDA;
    if (cudaGetSymbolAddress(&tables, g_noalloc_tables) != cudaSuccess) return SDFT_ERR_CUDA;
    if (cudaGetSymbolAddress(&w64, g_noalloc_w64) != cudaSuccess) return SDFT_ERR_CUDA;
    const KernelInfo* k15 = large_kernel(15);
    const KernelInfo* k16 = large_kernel(16);
    if (!k15 || !k16 || k15->tw_entries != kTw15 || k16->tw_entries != kTw16)
        return SDFT_ERR_UNSUPPORTED_N;
    if (k15->prepare() != cudaSuccess || k16->prepare() != cudaSuccess) return SDFT_ERR_CUDA;
    cudaStream_t st = nullptr;  // legacy default stream: ordered with everything on the device
    W64 host = {};
    if (make_w64(&host, static_cast<float2*>(w64), st) != cudaSuccess) return SDFT_ERR_CUDA;
    float2* base = static_cast<float2*>(tables);
    if (make_tables(base, k15->tables, k15->ntables, st) != cudaSuccess ||
        make_tables(base + kTw15, k16->tables, k16->ntables, st) != cudaSuccess)
        return SDFT_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return SDFT_ERR_CUDA;
    s.scratch = static_cast<float2*>(scratch);
    s.tables = base;
    s.w64 = host;
    s.ready = true;
    return SDFT_OK;
}

bool overlap(const void* a, const void* b, size_t bytes) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + bytes && y < x + bytes;
}

}  // namespace
}  // namespace sdft

extern "C" int sdft_execute_noalloc(int64_t n, int64_t batch, int direction, const float* xr,
                                    const float* xi, float* yr, float* yi, void* stream) {
    using namespace sdft;
    if (n != 32768 && n != 65536) return SDFT_ERR_UNSUPPORTED_N;   // only the scratch kernel
    if (batch < 1 || batch > ((int64_t)1 << 40) / n) return SDFT_ERR_INVALID_ARG;
    if (direction != SDFT_FORWARD && direction != SDFT_ADJOINT) return SDFT_ERR_INVALID_ARG;
    if (!xr || !xi || !yr || !yi) return SDFT_ERR_INVALID_ARG;
    const uintptr_t ptrs[4] = {(uintptr_t)xr, (uintptr_t)xi, (uintptr_t)yr, (uintptr_t)yi};
    for (uintptr_t p : ptrs)
        if (p % 16 != 0) return SDFT_ERR_MISALIGNED;
    const size_t bytes = (size_t)(n * batch) * sizeof(float);
    const bool in_place = (yr == xr) && (yi == xi);
    if (overlap(yr, yi, bytes)) return SDFT_ERR_ALIAS;
    if (in_place ? (overlap(yr, xi, bytes) || overlap(yi, xr, bytes))
                 : (overlap(yr, xr, bytes) || overlap(yr, xi, bytes) || overlap(yi, xr, bytes) ||
                    overlap(yi, xi, bytes)))
        return SDFT_ERR_ALIAS;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SDFT_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SDFT_ERR_INVALID_ARG;
    DeviceState state;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        const int s = setup(dev);
        if (s != SDFT_OK) return s;
        state = g_state[dev];
    }
    const int logn = n == 65536 ? 16 : 15;
    const KernelInfo* k = large_kernel(logn);
    const int64_t slots = kNoAllocScratch / n;
    LaunchArgs a;
    a.xr = xr;
    a.xi = xi;
    a.yr = yr;
    a.yi = yi;
    a.batch = batch;
    a.tw = state.tables + (logn == 16 ? kTw15 : 0);
    a.w64 = state.w64;
    a.scratch = state.scratch;
    a.status = nullptr;
    a.aux = nullptr;
    a.grid = (int)(batch < slots ? batch : slots);
    a.stream = (cudaStream_t)stream;
    a.adj = (direction == SDFT_ADJOINT);
    return k->launch(a) == cudaSuccess ? SDFT_OK : SDFT_ERR_CUDA;
}
