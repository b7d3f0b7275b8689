// kernels_large.cu -- planar FP32 DFT for N = 32768 and 65536.
//
// A transform this long (256 or 512 KiB of FP32 pairs) exceeds one SM's
// registers and shared memory, so each CTA runs its transform as two passes
// over a CTA-private scratch slot (N = A * C, n = col + C * ntop,
// k = d + A * k2):
//   pass 1: for every column col < C, an A-point DFT over ntop, rotated by
//           W_N^{col * d}, written to scratch[d][col];
//   pass 2: for every row d < A, a C-point DFT over col of scratch[d][.],
//           written to y[d + A * k2].
// This is the same regrouping of the radix-2 factors of Eq. (6) that the
// row kernels use, with one extra level.  A persistent grid of one CTA per SM
// keeps the scratch slots (N * 8 bytes each) resident in L2, so the extra
// round trip mostly stays on chip.  Each transform is read completely (pass
// 1) before any of its output is written (pass 2), so in-place calls are safe.
//
// Inside each pass the sub-DFTs are run by the step engine with lanes mapped
// to columns (pass 1) or rows (pass 2), so every global access of a warp is
// a contiguous 128-byte line per plane.
#include "kernels_large.cuh"

namespace sdft {

template <class CFG>
cudaError_t large_prepare() {
    cudaError_t e = cudaFuncSetAttribute(k_large<CFG, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CFG::SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_large<CFG, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)CFG::SMEM);
}

template <class CFG>
int large_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_large<CFG, false>, CFG::THREADS,
                                                      CFG::SMEM) != cudaSuccess)
        return 0;
    return n;
}

template <class CFG>
cudaError_t large_launch(const LaunchArgs& a) {
    if (a.adj)
        return launch_kernel(k_large<CFG, true>, a.grid, CFG::THREADS, CFG::SMEM, a.stream, a.xr,
                             a.xi, a.yr, a.yi, a.batch, a.tw, a.scratch, a.w64);
    return launch_kernel(k_large<CFG, false>, a.grid, CFG::THREADS, CFG::SMEM, a.stream, a.xr,
                         a.xi, a.yr, a.yi, a.batch, a.tw, a.scratch, a.w64);
}

template <class CFG>
KernelInfo large_info(const char* name) {
    using SA = typename CFG::SA_;
    using SC = typename CFG::SC_;
    KernelInfo k = {};
    k.name = name;
    k.logn = CFG::LOGN;
    k.threads = CFG::THREADS;
    k.smem = CFG::SMEM;
    k.transforms_per_cta = 1;
    k.ntables = 3;
    k.tables[0] = TableDesc{CFG::A, (int64_t)1 << SA::lr(0), (int64_t)CFG::A >> SA::lr(0), CFG::TWA};
    k.tables[1] = TableDesc{CFG::C, (int64_t)1 << SC::lr(0), (int64_t)CFG::C >> SC::lr(0), CFG::TWC};
    k.tables[2] = TableDesc{CFG::N, CFG::A, CFG::C, CFG::TWB};
    k.tw_entries = CFG::TW_TOTAL;
    k.scratch_per_cta = CFG::N;
    k.launches = 1;
    k.prepare = large_prepare<CFG>;
    k.blocks_per_sm = large_blocks_per_sm<CFG>;
    k.launch = large_launch<CFG>;
    return k;
}

const KernelInfo* large_kernel(int logn) {
    using S256 = Steps<8, 4, 4, 4, 0>;   // 16 threads x 16 values, radix [16,16]
    using S128 = Steps<7, 4, 4, 3, 0>;   // 8 threads x 16 values, radix [16,8]
    static const KernelInfo k15 = large_info<LargeCfgT<8, 7, S256, S128>>(
        "N=32768: two passes per CTA through L2-resident scratch, 256 x 128, radix [16,16]x[16,8]");
    static const KernelInfo k16 = large_info<LargeCfgT<8, 8, S256, S256>>(
        "N=65536: two passes per CTA through L2-resident scratch, 256 x 256, radix [16,16]x[16,16]");
    switch (logn) {
        case 15: return &k15;
        case 16: return &k16;
        default: return nullptr;
    }
}

}  // namespace sdft
