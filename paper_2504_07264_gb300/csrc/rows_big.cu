// rows_big.cu -- compiled row-kernel configurations for N = 2048 .. 16384:
// 32 complex values per thread, three register steps, two shared-memory
// exchanges; a transform spans 2 .. 16 warps of one CTA.
#include "kernels_rows.cuh"

namespace sdft {

const KernelInfo* rows_kernel_big(int logn) {
    static const KernelInfo k11 = rows_info<RowCfg<11, 5, 5, 4, 2, 4, 0, 2>>("N=2048: 64 threads/transform, radix [32,16,4]");
    static const KernelInfo k12 = rows_info<RowCfg<12, 5, 5, 5, 2, 2, 0, 2>>("N=4096: 128 threads/transform, radix [32,32,4]");
    static const KernelInfo k13 = rows_info<RowCfg<13, 5, 5, 5, 3, 1, 0, 2>>("N=8192: 256 threads/transform, radix [32,32,8]");
    static const KernelInfo k14 = rows_info<RowCfg<14, 5, 5, 5, 4, 1>>("N=16384: 512 threads/transform, radix [32,32,16]");
    switch (logn) {
        case 11: return &k11;
        case 12: return &k12;
        case 13: return &k13;
        case 14: return &k14;
        default: return nullptr;
    }
}

}  // namespace sdft
