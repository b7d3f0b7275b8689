// twiddle.cuh -- the float64 twiddle generator shared by the table kernels.
//
// W_M^e = exp(-j 2 pi e / M) is computed in float64 with sincospi on the
// first octant (argument 2r/M <= 1/4, an exact dyadic rational) and rounded
// once to float32; the other octants follow by exact swaps and sign changes,
// so W = 1, -j, -1, +j are exact and every table is exactly symmetric.  This
// is the only float64 arithmetic the library performs on the GPU.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sdft {

// (cos(2 pi e / M), -sin(2 pi e / M)) rounded to float32, M a power of two.
__device__ __forceinline__ float2 twiddle_value(int64_t e, int64_t M) {
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

}  // namespace sdft
