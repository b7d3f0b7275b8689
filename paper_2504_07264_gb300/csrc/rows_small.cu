// rows_small.cu -- compiled row-kernel configurations for N = 2 .. 512.
// Schedules: N <= 32 one thread per transform; N = 64 .. 512 two register
// steps and one shared-memory exchange (pad words chosen so the warps' two
// or four transforms fall on disjoint banks).
#include "kernels_rows.cuh"

namespace sdft {

const KernelInfo* rows_kernel_small(int logn) {
    //                                 LOGN LOGE  LR0 LR1 LR2   G  SBX
    static const KernelInfo k1 = rows_info<RowCfg<1, 1, 1, 0, 0, 256>>("N=2: 1 thread/transform, radix [2]");
    static const KernelInfo k2 = rows_info<RowCfg<2, 2, 2, 0, 0, 256>>("N=4: 1 thread/transform, radix [4]");
    static const KernelInfo k3 = rows_info<RowCfg<3, 3, 3, 0, 0, 256>>("N=8: 1 thread/transform, radix [8]");
    static const KernelInfo k4 = rows_info<RowCfg<4, 4, 4, 0, 0, 256>>("N=16: 1 thread/transform, radix [16]");
    static const KernelInfo k5 = rows_info<RowCfg<5, 5, 5, 0, 0, 128>>("N=32: 1 thread/transform, radix [32]");
    static const KernelInfo k6 = rows_info<RowCfg<6, 3, 3, 3, 0, 32, 2>>("N=64: 8 threads/transform, radix [8,8]");
    static const KernelInfo k7 = rows_info<RowCfg<7, 4, 4, 3, 0, 32>>("N=128: 8 threads/transform, radix [16,8]");
    static const KernelInfo k8 = rows_info<RowCfg<8, 4, 4, 4, 0, 16>>("N=256: 16 threads/transform, radix [16,16]");
    static const KernelInfo k9 = rows_info<RowCfg<9, 5, 5, 4, 0, 16, 16, 2>>("N=512: 16 threads/transform, radix [32,16]");
    switch (logn) {
        case 1: return &k1;
        case 2: return &k2;
        case 3: return &k3;
        case 4: return &k4;
        case 5: return &k5;
        case 6: return &k6;
        case 7: return &k7;
        case 8: return &k8;
        case 9: return &k9;
        default: return nullptr;
    }
}

}  // namespace sdft
