// rows_pf.cu -- row-kernel candidates whose input tiles are prefetched by
// 1-D bulk copies (k_rows_pf): 128-thread CTAs of 4096 points, three per SM
// (N = 512 .. 4096), one or two 256-thread CTAs per SM (N = 8192; with two, a
// quarter or half of each next row in shared memory and the rest prefetched
// into L2), or one 512-thread CTA per SM with half of each row in shared
// memory and half in L2 (N = 16384).
// (For N = 64 .. 256 and 1024 the same form measured slower than the
// 256-thread kernels, which stay the only candidates there.)
// N = 4096 .. 16384 exchange through the XOR-swizzled layout (swz32), which
// takes exactly N words per plane: the CTAs' shared memory then fits the 196
// KiB carveout instead of the 228 KiB one (3 x 64 KiB at N = 4096, 2 x 96 KiB
// at N = 8192, 192 KiB at N = 16384), which leaves 60 KiB of L1 instead of 28
// for the rotation tables and the lines read from L2 (bank conflicts stay
// about the same): 381 -> 399 (4096), 334 -> 347 (8192) and 292 -> 309 Gpts/s
// (16384).  N = 2048 (radix [32,16,4], two transforms per tile) keeps the
// padded layout: swizzled it also fits the smaller carveout but measured 376
// against 387.  (Other radix orders of the swizzled half-row forms measured
// slower: N = 8192 [32,16,16] 335, [16,32,16] 329, [8,32,32] 319 against 351,
// Eq. (6) order 348; N = 16384 [32,16,32] 299, [16,32,32] 295 against 311;
// N = 16384 in Eq. (6) order 317, kept as a candidate.)  With the exchange at exactly N words,
// three quarters of the next row also fit (N = 8192: two CTAs per SM; N =
// 16384: 224 KiB): 345 and 305 against 351 and 310 for half a row.
#include "kernels_rows.cuh"

namespace sdft {

const KernelInfo* rows_pf_candidate(int logn, int idx) {
    //                                           LOGN LOGE LR0 LR1 LR2  G
    static const KernelInfo k9 = rows_pf_info<RowPfCfg<RowCfg<9, 5, 5, 4, 0, 8>>>(
        "N=512: 16 threads/transform, radix [32,16], input tiles prefetched by TMA");
    static const KernelInfo k11 = rows_pf_info<RowPfCfg<RowCfg<11, 5, 5, 4, 2, 2>>>(
        "N=2048: 64 threads/transform, radix [32,16,4], input tiles prefetched by TMA");
    static const KernelInfo k12 = rows_pf_info<RowPfCfg<RowCfg<12, 5, 5, 5, 2, 1, 0, 1, false, true>>>(
        "N=4096: 128 threads/transform, radix [32,32,4], input tiles prefetched by TMA, swizzled exchange");
    // one 8192-point transform per 256-thread CTA: 130 KiB of shared memory,
    // so one CTA per SM, its next transform always in flight
    static const KernelInfo k13 = rows_pf_info<RowPfCfg<RowCfg<13, 5, 5, 5, 3, 1, 0, 1, false, true>, 1>>(
        "N=8192: 256 threads/transform, radix [32,32,8], input tiles prefetched by TMA, swizzled exchange");
    // one 16384-point transform per 512-thread CTA, half of the next row in
    // flight in shared memory (the whole row does not fit beside the exchange
    // buffer) and the other half prefetched into L2
    static const KernelInfo k14 = rows_pf_info<RowPfCfg<RowCfg<14, 5, 5, 5, 4, 1, 0, 1, false, true>, 1, 2>>(
        "N=16384: 512 threads/transform, radix [32,32,16], half of each input row prefetched by TMA, "
        "swizzled exchange");
    // two 8192-point CTAs per SM, half or a quarter of the next row in
    // flight in shared memory, the rest of it prefetched into L2
    static const KernelInfo k13h = rows_pf_info<RowPfCfg<RowCfg<13, 5, 5, 5, 3, 1, 0, 1, false, true>, 2, 2>>(
        "N=8192: 256 threads/transform, radix [32,32,8], half of each input row prefetched by TMA, "
        "two CTAs/SM, swizzled exchange");
    static const KernelInfo k13q = rows_pf_info<RowPfCfg<RowCfg<13, 5, 5, 5, 3, 1, 0, 1, false, true>, 2, 4>>(
        "N=8192: 256 threads/transform, radix [32,32,8], a quarter of each input row prefetched by "
        "TMA, two CTAs/SM, swizzled exchange");
    // the same in the order of Eq. (6) (bit-reversed gathers, D(i) then W(i))
    static const KernelInfo k14d = rows_pf_info<RowPfCfg<RowCfg<14, 5, 5, 5, 4, 1, 0, 1, true, true>, 1, 2>>(
        "N=16384: 512 threads/transform, radix [32,32,16], Eq. (6) order, half of each input row "
        "prefetched by TMA, swizzled exchange");
    if (logn == 14 && idx == 1) return &k14d;
    if (logn == 13 && idx == 1) return &k13h;
    if (logn == 13 && idx == 2) return &k13q;
    if (idx != 0) return nullptr;
    switch (logn) {
        case 9: return &k9;
        case 11: return &k11;
        case 12: return &k12;
        case 13: return &k13;
        case 14: return &k14;
        default: return nullptr;
    }
}

}  // namespace sdft
