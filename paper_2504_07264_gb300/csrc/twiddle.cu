// twiddle.cu -- twiddle-factor tables for the planar DFT kernels.
//
// Every rotation factor is W_M^e = exp(-j 2 pi e / M) = cos(2 pi e / M)
// - j sin(2 pi e / M), the entries of the 2x2 blocks omega^(i,q) of Section III
// (definitions under Eq. (6)) generalised to the regrouped steps.  Values are
// computed in float64 on the device with sincospi on the first octant
// (argument 2r/M <= 1/4, an exact dyadic rational) and rounded once to
// float32; the other octants follow by exact swaps and sign changes, so
// W = 1, -j, -1, +j are exact and the table is exactly symmetric.  This is
// the only float64 arithmetic the library performs on the GPU.
#include "launch.h"
#include "twiddle.cuh"

namespace sdft {

__global__ void k_table(float2* dst, TableDesc d) {
    const int64_t n = d.R * d.Q;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t dd = u / d.Q, nl = u % d.Q;
        dst[d.offset + u] = twiddle_value((nl * dd) % d.M, d.M);
    }
}

__global__ void k_w64(float2* dst) {
    const int q = threadIdx.x;
    if (q < 64) dst[q] = twiddle_value(q, 64);
}

cudaError_t make_tables(float2* dst, const TableDesc* desc, int count, cudaStream_t stream) {
    for (int i = 0; i < count; ++i) {
        const int64_t n = desc[i].R * desc[i].Q;
        if (n <= 0) continue;
        const int threads = 256;
        const int64_t blocks64 = (n + threads - 1) / threads;
        const int blocks = (int)(blocks64 < 4096 ? blocks64 : 4096);
        cudaError_t e = launch_kernel(k_table, blocks, threads, 0, stream, dst, desc[i]);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t make_w64(W64* w64, float2* scratch64, cudaStream_t stream) {
    cudaError_t e = launch_kernel(k_w64, 1, 64, 0, stream, scratch64);
    if (e != cudaSuccess) return e;
    float2 host[64];
    e = cudaMemcpyAsync(host, scratch64, sizeof(host), cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return e;
    for (int q = 0; q < 64; ++q) {
        w64->c[q] = host[q].x;
        w64->s[q] = host[q].y;
    }
    return cudaSuccess;
}

}  // namespace sdft
