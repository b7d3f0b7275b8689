// rows_big.cu -- compiled row-kernel candidates for N = 2048 .. 16384: three
// register steps and two shared-memory exchanges; a transform spans 2 .. 16
// warps of one CTA.  Candidate 0 holds 32 complex values per thread; the
// 16-value candidates trade a lower register count for more resident warps.
#include "kernels_rows.cuh"

namespace sdft {

const KernelInfo* rows_candidate_big(int logn, int idx) {
    static const KernelInfo k11[] = {
        rows_info<RowCfg<11, 5, 5, 4, 2, 4, 0, 2>>("N=2048: 64 threads/transform, radix [32,16,4]"),
        rows_info<RowCfg<11, 4, 4, 4, 3, 2, 0, 4>>("N=2048: 128 threads/transform, radix [16,16,8]"),
        rows_info<RowCfg<11, 5, 5, 4, 2, 4, 0, 2, true>>("N=2048: 64 threads/transform, radix [32,16,4], Eq. (6) order")};
    static const KernelInfo k12[] = {
        rows_info<RowCfg<12, 5, 5, 5, 2, 2, 0, 2>>("N=4096: 128 threads/transform, radix [32,32,4]"),
        rows_info<RowCfg<12, 4, 4, 4, 4, 1, 0, 4>>("N=4096: 256 threads/transform, radix [16,16,16]"),
        rows_info<RowCfg<12, 4, 4, 4, 4, 2, 0, 2>>("N=4096: 256 threads/transform, radix [16,16,16], 512-thread CTAs"),
        rows_info<RowCfg<12, 5, 5, 5, 2, 2, 0, 2, true>>("N=4096: 128 threads/transform, radix [32,32,4], Eq. (6) order")};
    static const KernelInfo k13[] = {
        rows_info<RowCfg<13, 5, 5, 5, 3, 1, 0, 2>>("N=8192: 256 threads/transform, radix [32,32,8]"),
        rows_info<RowCfg<13, 5, 5, 4, 4, 1, 0, 2>>("N=8192: 256 threads/transform, radix [32,16,16]"),
        rows_info<RowCfg<13, 5, 5, 5, 3, 1, 0, 2, true>>("N=8192: 256 threads/transform, radix [32,32,8], Eq. (6) order")};
    static const KernelInfo k14[] = {
        rows_info<RowCfg<14, 5, 5, 5, 4, 1>>("N=16384: 512 threads/transform, radix [32,32,16]"),
        rows_info<RowCfg<14, 5, 5, 5, 4, 1, 0, 1, true>>("N=16384: 512 threads/transform, radix [32,32,16], Eq. (6) order")};
#define SDFT_PICK(arr) return idx < (int)(sizeof(arr) / sizeof(arr[0])) ? &arr[idx] : nullptr
    if (idx < 0) return nullptr;
    switch (logn) {
        case 11: SDFT_PICK(k11);
        case 12: SDFT_PICK(k12);
        case 13: SDFT_PICK(k13);
        case 14: SDFT_PICK(k14);
        default: return nullptr;
    }
#undef SDFT_PICK
}

// After the prefetching candidates: N = 8192 as 128 threads x 64 values with
// an XOR-swizzled exchange of exactly 64 KiB, three CTAs per SM (24 K points in
// flight per SM; measured 285 against 333 Gpts/s for the quarter-row prefetch).
const KernelInfo* rows_candidate_e64(int logn, int idx) {
    static const KernelInfo k13 = rows_info<RowCfg<13, 6, 5, 5, 3, 1, 0, 3, false, true>>(
        "N=8192: 128 threads x 64 values/transform, radix [32,32,8], swizzled exchange, "
        "three CTAs/SM");
    return (logn == 13 && idx == 0) ? &k13 : nullptr;
}

}  // namespace sdft
