// launch.h -- internal interface between the C ABI (sdft_api.cu) and the
// kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "fft_core.cuh"

namespace sdft {

// One twiddle table: entries tab[offset + d * Q + nl] = W_M^{(nl * d) mod M}
// for d < R, nl < Q (M a power of two).
struct TableDesc {
    int64_t M, R, Q, offset;
};

struct LaunchArgs {
    const float* xr;
    const float* xi;
    float* yr;
    float* yi;
    long long batch;        // transforms (uniform plans)
    const float2* tw;       // device twiddle tables of the kernel
    W64 w64;                // register-DFT constants
    float2* scratch;        // per-CTA scratch (kernels that need it), else null
    int* status;            // device status word
    const void* aux;        // kernel-specific constant data (split path: block matrices)
    int grid;               // CTAs to launch
    cudaStream_t stream;
    bool adj;
};

// A compiled kernel configuration for one transform length.
struct KernelInfo {
    const char* name;            // human-readable schedule
    int logn;                    // log2 N
    int threads;                 // threads per CTA
    size_t smem;                 // dynamic shared memory per CTA (bytes)
    int transforms_per_cta;      // transforms one CTA processes per tile
    int ntables;                 // twiddle tables used
    TableDesc tables[4];
    int64_t tw_entries;          // float2 entries over all tables
    int64_t scratch_per_cta;     // float2 scratch entries per resident CTA (0 = none)
    int launches;                // kernel launches per call
    bool queue;                  // run as items of the persistent work-queue kernel
    int cluster;                 // CTAs per thread-block cluster (0: no clusters)
    cudaError_t (*prepare)();    // one-time function attributes
    int (*blocks_per_sm)();      // occupancy of the kernel
    int (*resident_ctas)();      // cluster kernels: CTAs resident over the GPU (else null)
    cudaError_t (*launch)(const LaunchArgs&);
};

// Tables of compiled configurations (defined by the kernel units).
const KernelInfo* rows_kernel(int logn);      // N = 2 .. 16384, one kernel
const KernelInfo* large_kernel(int logn);     // N = 32768, 65536
const KernelInfo* cluster_kernel(int logn, int idx);   // N = 16384 .. 65536, one cluster per transform

// Twiddle generation (twiddle.cu): fill `count` descriptors into `dst`
// (device), and the 64-entry register constant table into `w64`.
cudaError_t make_tables(float2* dst, const TableDesc* desc, int count, cudaStream_t stream);
cudaError_t make_w64(W64* w64, float2* scratch64, cudaStream_t stream);

// Launch helper: one kernel through cudaLaunchKernelEx so the launch status is
// returned directly rather than read from the sticky last-error slot.
template <typename... KArgs, typename... Act>
inline cudaError_t launch_kernel(void (*kern)(KArgs...), int grid, int threads, size_t smem,
                                 cudaStream_t stream, Act&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cfg.attrs = nullptr;
    cfg.numAttrs = 0;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<Act&&>(args)...);
}

}  // namespace sdft
