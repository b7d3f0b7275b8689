// rows_1024.cu -- compiled row-kernel configuration for N = 1024: one warp
// per transform, radix [32, 32] (32 complex values per lane), one padded
// shared-memory exchange between the two register steps.
#include "kernels_rows.cuh"

namespace sdft {

const KernelInfo* rows_kernel_1024(int logn) {
    static const KernelInfo k10 = rows_info<RowCfg<10, 5, 5, 5, 0, 8, 0, 2>>("N=1024: 32 threads/transform, radix [32,32]");
    return logn == 10 ? &k10 : nullptr;
}

}  // namespace sdft
