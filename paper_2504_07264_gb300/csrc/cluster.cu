// cluster.cu -- the uniform cluster kernel for N = 16384 .. 65536: one
// thread-block cluster of N / 8192 CTAs per transform (kernels_cluster.cuh;
// N = 32768 also as N / 4096 CTAs of 128 threads), two (four) CTAs of
// different clusters per SM, a persistent grid: cluster c
// handles transforms c, c + (clusters), ...  Pass 1 loads straight into
// registers and pass 2 stores straight from registers.
#include "kernels_cluster.cuh"
#include "launch.h"

namespace sdft {
namespace {

template <class CFG, bool ADJ>
__global__ void __launch_bounds__(CFG::THREADS, CFG::MINB)
k_cluster(const float* __restrict__ xr, const float* __restrict__ xi, float* __restrict__ yr,
          float* __restrict__ yi, const long long batch, const float2* __restrict__ tw,
          const W64 w) {
    constexpr int A = CFG::A, C = CFG::C, CQ = CFG::CQ, AQ = CFG::AQ;
    extern __shared__ float4 smem4[];
    float* const work = reinterpret_cast<float*>(smem4);
    const uint32_t y_sh = (uint32_t)__cvta_generic_to_shared(work);
    const int tid = (int)threadIdx.x;
    const uint32_t rank = cluster_ctarank();
    const int col = (int)rank * CQ + tid % CQ;
    const int d = (int)rank * AQ + tid % AQ;
    constexpr uint32_t SHARE = (uint32_t)(CFG::N / CFG::Q) * 4u;   // bytes per plane per CTA
    for (long long t = cluster_id(); t < batch; t += cluster_count()) {
        const float* gxr = xr + t * CFG::N;
        const float* gxi = xi + t * CFG::N;
        // the cluster's next transform into L2 while this one runs (each CTA
        // one contiguous share of each plane)
        const long long tn = t + cluster_count();
        if (tid == 0 && tn < batch) {
            prefetch_l2(xr + tn * CFG::N + (long long)rank * (CFG::N / CFG::Q), SHARE);
            prefetch_l2(xi + tn * CFG::N + (long long)rank * (CFG::N / CFG::Q), SHARE);
        }
        auto ld = [&](int L, float& r, float& i) {
            r = gxr[col + C * L];
            i = gxi[col + C * L];
        };
        pass1<CFG, ADJ>(ld, [] {}, work, tid, col, tw, w);
        cluster_arrive();   // Y of this CTA complete (release) ...
        cluster_wait();     // ... and of every CTA of the cluster (acquire)
        float* const gyr = yr + t * CFG::N;
        float* const gyi = yi + t * CFG::N;
        auto st = [&](int k2, float r, float i) {
            __stcs(gyr + d + A * k2, r);   // evict-first: keeps L2 for the prefetched input
            __stcs(gyi + d + A * k2, i);
        };
        pass2<CFG, ADJ>(st, work, y_sh, tid, d, 0, tw, w);
    }
}

template <class CFG>
cudaError_t cluster_prepare() {
    for (const void* f : {(const void*)k_cluster<CFG, false>, (const void*)k_cluster<CFG, true>}) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)CFG::SMEM);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <class CFG>
cudaLaunchConfig_t cluster_config(int grid, cudaStream_t stream, cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3((unsigned)CFG::THREADS, 1, 1);
    cfg.dynamicSmemBytes = CFG::SMEM;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CFG::Q;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

// CTAs resident at once over the whole GPU: the occupancy query for clusters
// (it accounts for how clusters fit the GPCs), times the cluster size.
template <class CFG>
int cluster_resident_ctas() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = cluster_config<CFG>(CFG::Q * CFG::MINB * sms, nullptr, attr);
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_cluster<CFG, false>, &cfg) != cudaSuccess)
        return 0;
    return clusters * CFG::Q;
}

template <class CFG>
int cluster_blocks_per_sm() {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_cluster<CFG, false>, CFG::THREADS,
                                                      CFG::SMEM) != cudaSuccess)
        return 0;
    return n;
}

template <class CFG>
cudaError_t cluster_launch(const LaunchArgs& a) {
    int clusters = a.grid / CFG::Q;
    if (clusters < 1) clusters = 1;
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = cluster_config<CFG>(clusters * CFG::Q, a.stream, attr);
    if (a.adj)
        return cudaLaunchKernelEx(&cfg, k_cluster<CFG, true>, a.xr, a.xi, a.yr, a.yi, a.batch,
                                  a.tw, a.w64);
    return cudaLaunchKernelEx(&cfg, k_cluster<CFG, false>, a.xr, a.xi, a.yr, a.yi, a.batch, a.tw,
                              a.w64);
}

template <class CFG>
KernelInfo cluster_info(const char* name) {
    using SA = typename CFG::SA_;
    using SC = typename CFG::SC_;
    KernelInfo k = {};
    k.name = name;
    k.logn = CFG::LOGN;
    k.threads = CFG::THREADS;
    k.smem = CFG::SMEM;
    k.transforms_per_cta = 1;
    k.cluster = CFG::Q;
    k.ntables = 4;
    k.tables[0] = TableDesc{CFG::A, (int64_t)1 << SA::lr(0), (int64_t)CFG::A >> SA::lr(0), CFG::TWA};
    k.tables[1] = TableDesc{CFG::C, (int64_t)1 << SC::lr(0), (int64_t)CFG::C >> SC::lr(0), CFG::TWC};
    k.tables[2] = TableDesc{CFG::N, CFG::P, CFG::C, CFG::TWB1};
    k.tables[3] = TableDesc{CFG::N / CFG::P, CFG::R1, CFG::C, CFG::TWB2};
    k.tw_entries = CFG::TW_TOTAL;
    k.scratch_per_cta = 0;
    k.launches = 1;
    k.prepare = cluster_prepare<CFG>;
    k.blocks_per_sm = cluster_blocks_per_sm<CFG>;
    k.resident_ctas = cluster_resident_ctas<CFG>;
    k.launch = cluster_launch<CFG>;
    return k;
}

}  // namespace

const KernelInfo* cluster_kernel(int logn, int idx) {
    static const KernelInfo k14 = cluster_info<Cluster14>(
        "N=16384: cluster of 2 CTAs, distributed shared memory, 128 x 128, radix [32,4]x[32,4]");
    static const KernelInfo k15 = cluster_info<Cluster15>(
        "N=32768: cluster of 4 CTAs, distributed shared memory, 256 x 128, radix [32,8]x[32,4]");
    static const KernelInfo k16 = cluster_info<Cluster16>(
        "N=65536: cluster of 8 CTAs, distributed shared memory, 256 x 256, radix [32,8]x[32,8]");
    static const KernelInfo k15q = cluster_info<Cluster15q>(
        "N=32768: cluster of 8 CTAs of 128 threads, distributed shared memory, 256 x 128, "
        "radix [32,8]x[32,4]");
    static const KernelInfo k16e = cluster_info<Cluster16e>(
        "N=65536: cluster of 8 CTAs of 128 threads x 64 values, three per SM, distributed "
        "shared memory, 256 x 256, radix [32,8]x[32,8]");
    static const KernelInfo k15e = cluster_info<Cluster15e>(
        "N=32768: cluster of 4 CTAs of 128 threads x 64 values, three per SM, distributed "
        "shared memory, 256 x 128, radix [32,8]x[16,8]");
    static const KernelInfo k14e = cluster_info<Cluster14e>(
        "N=16384: cluster of 2 CTAs of 128 threads x 64 values, three per SM, distributed "
        "shared memory, 128 x 128, radix [16,8]x[16,8]");
    if (logn == 15 && idx == 1) return &k15q;
    if (logn == 16 && idx == 1) return &k16e;
    if (logn == 15 && idx == 2) return &k15e;
    if (logn == 14 && idx == 1) return &k14e;
    if (idx != 0) return nullptr;
    switch (logn) {
        case 14: return &k14;
        case 15: return &k15;
        case 16: return &k16;
        default: return nullptr;
    }
}

}  // namespace sdft
