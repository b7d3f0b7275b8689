// rows_small.cu -- compiled row-kernel candidates for N = 2 .. 512.
// Candidate 0 of each length is the default schedule: N <= 32 one thread per
// transform; N = 64 .. 512 two register steps and one shared-memory exchange
// (pad words chosen so the warps' two or four transforms fall on disjoint
// banks).  The other candidates change the radix split, the threads per
// transform, the register-DFT order (Eq. (6) order, "DIT") or, for N = 16
// and 32, move the rows through shared memory by whole lines (k_rows_tr);
// for N = 16 .. 64 the last one spreads a transform over 2 .. 8 lanes with
// butterflies across lanes by warp shuffles (k_rows_shfl).  The autotuner
// times them.
#include "kernels_rows.cuh"
#include "rows_shfl.h"

namespace sdft {

const KernelInfo* rows_candidate_small(int logn, int idx) {
    //                                  LOGN LOGE LR0 LR1 LR2  G  SBX MINB DIT
    static const KernelInfo k1[] = {
        rows_info<RowCfg<1, 1, 1, 0, 0, 256>>("N=2: 1 thread/transform, radix [2]"),
        rows_info<RowCfg<1, 1, 1, 0, 0, 256, 0, 1, true>>("N=2: 1 thread/transform, radix [2], Eq. (6) order")};
    static const KernelInfo k2[] = {
        rows_info<RowCfg<2, 2, 2, 0, 0, 256>>("N=4: 1 thread/transform, radix [4]"),
        rows_info<RowCfg<2, 2, 2, 0, 0, 256, 0, 1, true>>("N=4: 1 thread/transform, radix [4], Eq. (6) order")};
    static const KernelInfo k3[] = {
        rows_info<RowCfg<3, 3, 3, 0, 0, 256>>("N=8: 1 thread/transform, radix [8]"),
        rows_info<RowCfg<3, 3, 3, 0, 0, 256, 0, 1, true>>("N=8: 1 thread/transform, radix [8], Eq. (6) order")};
    static const KernelInfo k4[] = {
        rows_info<RowCfg<4, 4, 4, 0, 0, 256>>("N=16: 1 thread/transform, radix [16]"),
        rows_info<RowCfg<4, 4, 4, 0, 0, 256, 0, 1, true>>("N=16: 1 thread/transform, radix [16], Eq. (6) order"),
        rows_info<RowCfg<4, 2, 2, 2, 0, 64, 3>>("N=16: 4 threads/transform, radix [4,4]"),
        rows_tr_info<RowTrCfg<RowCfg<4, 4, 4, 0, 0, 256>>>(
            "N=16: 1 thread/transform, radix [16], rows moved by whole lines through shared memory")};
    static const KernelInfo k5[] = {
        rows_info<RowCfg<5, 5, 5, 0, 0, 128>>("N=32: 1 thread/transform, radix [32]"),
        rows_info<RowCfg<5, 5, 5, 0, 0, 128, 0, 1, true>>("N=32: 1 thread/transform, radix [32], Eq. (6) order"),
        rows_info<RowCfg<5, 3, 3, 2, 0, 64, 1>>("N=32: 4 threads/transform, radix [8,4]"),
        rows_tr_info<RowTrCfg<RowCfg<5, 5, 5, 0, 0, 128>>>(
            "N=32: 1 thread/transform, radix [32], rows moved by whole lines through shared memory")};
    static const KernelInfo k6[] = {
        rows_info<RowCfg<6, 3, 3, 3, 0, 32, 2>>("N=64: 8 threads/transform, radix [8,8]"),
        rows_info<RowCfg<6, 3, 3, 3, 0, 32, 2, 1, true>>("N=64: 8 threads/transform, radix [8,8], Eq. (6) order")};
    static const KernelInfo k7[] = {
        rows_info<RowCfg<7, 4, 4, 3, 0, 32>>("N=128: 8 threads/transform, radix [16,8]"),
        rows_info<RowCfg<7, 4, 4, 3, 0, 32, 0, 1, true>>("N=128: 8 threads/transform, radix [16,8], Eq. (6) order")};
    static const KernelInfo k8[] = {
        rows_info<RowCfg<8, 4, 4, 4, 0, 16>>("N=256: 16 threads/transform, radix [16,16]"),
        rows_info<RowCfg<8, 4, 4, 4, 0, 16, 0, 1, true>>("N=256: 16 threads/transform, radix [16,16], Eq. (6) order"),
        rows_info<RowCfg<8, 5, 5, 3, 0, 32, 8, 2>>("N=256: 8 threads/transform, radix [32,8]")};
    static const KernelInfo k9[] = {
        rows_info<RowCfg<9, 5, 5, 4, 0, 16, 16, 2>>("N=512: 16 threads/transform, radix [32,16]"),
        rows_info<RowCfg<9, 5, 5, 4, 0, 16, 16, 2, true>>("N=512: 16 threads/transform, radix [32,16], Eq. (6) order"),
        rows_info<RowCfg<9, 4, 4, 4, 1, 8, 0, 4>>("N=512: 32 threads/transform, radix [16,16,2]")};
    // after a length's own candidates: the warp-shuffle form (rows_shfl.cu)
#define SDFT_PICK(arr)                                                              \
    return idx < (int)(sizeof(arr) / sizeof(arr[0]))                               \
               ? &arr[idx]                                                          \
               : rows_shfl_candidate(logn, idx - (int)(sizeof(arr) / sizeof(arr[0])))
    if (idx < 0) return nullptr;
    switch (logn) {
        case 1: SDFT_PICK(k1);
        case 2: SDFT_PICK(k2);
        case 3: SDFT_PICK(k3);
        case 4: SDFT_PICK(k4);
        case 5: SDFT_PICK(k5);
        case 6: SDFT_PICK(k6);
        case 7: SDFT_PICK(k7);
        case 8: SDFT_PICK(k8);
        case 9: SDFT_PICK(k9);
        default: return nullptr;
    }
#undef SDFT_PICK
}

}  // namespace sdft
