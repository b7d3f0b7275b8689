// rows_1024.cu -- compiled row-kernel candidates for N = 1024.  Candidate 0:
// one warp per transform, radix [32, 32] (32 complex values per lane), one
// padded shared-memory exchange between the two register steps.  (Measured and
// left out: 16 threads x 64 values per transform, eight transforms per CTA of
// 128 threads, three CTAs per SM on a 64 KiB XOR-swizzled exchange whose
// rotation flips by 16 banks for odd transforms: 297 against 402 Gpts/s; and
// candidate 0 with thread 0 bringing the CTA's next tile into L2 by two bulk
// prefetches at the top of each tile: 325 against 402; and candidate 0 with
// each warp staging its next row into its own exchange buffer by 16-byte
// cp.async copies once step 1 has read it, step 0 then reading shared memory:
// 352 against 402.)
#include "kernels_rows.cuh"

namespace sdft {

const KernelInfo* rows_candidate_1024(int logn, int idx) {
    static const KernelInfo k10[] = {
        rows_info<RowCfg<10, 5, 5, 5, 0, 8, 0, 2>>("N=1024: 32 threads/transform, radix [32,32]"),
        rows_info<RowCfg<10, 5, 5, 5, 0, 8, 0, 2, true>>("N=1024: 32 threads/transform, radix [32,32], Eq. (6) order"),
        rows_info<RowCfg<10, 5, 5, 5, 0, 4, 0, 4>>("N=1024: 32 threads/transform, radix [32,32], 128-thread CTAs"),
        rows_info<RowCfg<10, 4, 4, 3, 3, 4, 0, 4>>("N=1024: 64 threads/transform, radix [16,8,8]"),
        rows_info<RowCfg<10, 4, 4, 4, 2, 4, 0, 4>>("N=1024: 64 threads/transform, radix [16,16,4]")};
    if (logn != 10 || idx < 0 || idx >= (int)(sizeof(k10) / sizeof(k10[0]))) return nullptr;
    return &k10[idx];
}

}  // namespace sdft
