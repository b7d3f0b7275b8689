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

namespace sdft {

// (cos(2 pi e / M), -sin(2 pi e / M)) rounded to float32, M a power of two.
__device__ float2 twiddle_value(int64_t e, int64_t M) {
    e %= M;
    if (e < 0) e += M;
    if (M < 8) {                          // only quarter turns are possible
        const int64_t q4 = (e * 4) / M;   // exact: M in {1, 2, 4}
        const float c[4] = {1.f, 0.f, -1.f, 0.f};
        const float s[4] = {0.f, 1.f, 0.f, -1.f};
        return make_float2(c[q4 & 3], -s[q4 & 3]);
    }
    const int64_t quarter = M / 4, eighth = M / 8;
    const int64_t quad = e / quarter;     // which quarter turn
    int64_t r = e % quarter;              // remainder angle 2 pi r / M < pi/2
    const bool swap = r > eighth;         // use the complementary angle
    if (swap) r = quarter - r;
    double sd, cd;
    sincospi((double)(2 * r) / (double)M, &sd, &cd);
    float cf = __double2float_rn(cd), sf = __double2float_rn(sd);
    if (r == eighth) sf = cf;             // 45 degrees: identical by construction
    if (swap) { const float t = cf; cf = sf; sf = t; }
    // rotate (cos, sin) of the remainder by quad quarter turns
    float c, s;
    switch (quad & 3) {
        case 0: c = cf; s = sf; break;
        case 1: c = -sf; s = cf; break;
        case 2: c = -cf; s = -sf; break;
        default: c = sf; s = -cf; break;
    }
    return make_float2(c, -s);
}

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
