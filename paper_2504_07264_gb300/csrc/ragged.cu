// ragged.cu -- host side of the persistent work-queue kernel
// (ragged_kernel.cuh): the compiled forms of every length class, launch
// attributes and occupancy.
#include "ragged.h"
#include "ragged_kernel.cuh"

namespace sdft {
const void* ragged_kernel_fwd();
const void* ragged_kernel_adj();

namespace {

using namespace rq;

template <class CFG>
RaggedForm row_form(const char* name, int code) {
    RaggedForm f = {};
    f.name = name;
    f.code = code;
    f.logn = CFG::S::LOGN;
    f.q = 1;
    f.per_item = CFG::G;
    f.ntables = rows_tables<CFG>(f.tables);
    f.tw_entries = CFG::TW_TOTAL;
    return f;
}

template <class CFG>
RaggedForm group_form(const char* name, int code) {
    using SA = typename CFG::SA_;
    using SC = typename CFG::SC_;
    RaggedForm f = {};
    f.name = name;
    f.code = code;
    f.logn = CFG::LOGN;
    f.q = CFG::Q;
    f.per_item = 1;
    f.ntables = 4;
    f.tables[0] = TableDesc{CFG::A, (int64_t)1 << SA::lr(0), (int64_t)CFG::A >> SA::lr(0), CFG::TWA};
    f.tables[1] = TableDesc{CFG::C, (int64_t)1 << SC::lr(0), (int64_t)CFG::C >> SC::lr(0), CFG::TWC};
    f.tables[2] = TableDesc{CFG::N, CFG::P, CFG::C, CFG::TWB1};
    f.tables[3] = TableDesc{CFG::N / CFG::P, CFG::R1, CFG::C, CFG::TWB2};
    f.tw_entries = CFG::TW_TOTAL;
    return f;
}

struct FormTable {
    RaggedForm f[17][4];
    int count[17];
};

const FormTable& forms() {
    static const FormTable t = [] {
        FormTable x = {};
        auto add = [&](const RaggedForm& f) { x.f[f.logn][x.count[f.logn]++] = f; };
        // form 0 of each length is the default
        add(row_form<R2>("N=4: tile of 128 transforms, 1 thread each", kR2));
        add(row_form<R3>("N=8: tile of 128 transforms, 1 thread each", kR3));
        add(row_form<R4>("N=16: tile of 128 transforms, 1 thread each", kR4));
        add(row_form<R5>("N=32: tile of 128 transforms, 1 thread each, radix [32]", kR5));
        add(row_form<R6>("N=64: tile of 16 transforms, 8 threads each, radix [8,8]", kR6));
        add(row_form<R7>("N=128: tile of 16 transforms, 8 threads each, radix [16,8]", kR7));
        add(row_form<R8>("N=256: tile of 8 transforms, 16 threads each, radix [16,16]", kR8));
        add(row_form<R8b>("N=256: tile of 16 transforms, 8 threads x 32 values, radix [32,8]", kR8b));
        add(row_form<R9>("N=512: tile of 8 transforms, 16 threads each, radix [32,16]", kR9));
        add(row_form<R9b>("N=512: tile of 4 transforms, 32 threads each, radix [16,16,2]", kR9b));
        add(row_form<R10>("N=1024: tile of 4 transforms, 32 threads each, radix [32,32]", kR10));
        add(row_form<R10b>("N=1024: tile of 2 transforms, 64 threads each, radix [16,8,8]", kR10b));
        add(row_form<R11>("N=2048: tile of 2 transforms, 64 threads each, radix [32,16,4]", kR11));
        add(row_form<R11b>("N=2048: tile of 1 transform, 128 threads, radix [16,16,8]", kR11b));
        add(row_form<R12>("N=4096: tile of 1 transform, 128 threads, radix [32,32,4]", kR12));
        add(group_form<Cluster13>("N=8192: 2 CTAs per transform, distributed shared memory, 128 x 64", kC13));
        add(group_form<Cluster14q>("N=16384: 4 CTAs x 32 values per thread, distributed shared memory, 128 x 128", kC14q));
        add(group_form<Cluster15q>("N=32768: 8 CTAs x 32 values per thread, distributed shared memory, 256 x 128", kC15q));
        add(group_form<Cluster16e>("N=65536: 8 CTAs x 64 values per thread, distributed shared memory, 256 x 256", kC16e));
        return x;
    }();
    return t;
}

}  // namespace

int ragged_form_count(int logn) { return (logn >= 2 && logn <= 16) ? forms().count[logn] : 0; }

const RaggedForm* ragged_form(int logn, int f) {
    if (f < 0 || f >= ragged_form_count(logn)) return nullptr;
    return &forms().f[logn][f];
}

int ragged_threads() { return kThreads; }
size_t ragged_smem() { return kSmem; }

const void* ragged_kernel_fn(bool adj) { return adj ? ragged_kernel_adj() : ragged_kernel_fwd(); }

cudaError_t ragged_prepare() {
    for (const void* f : {ragged_kernel_fwd(), ragged_kernel_adj()}) {
        const cudaError_t e =
            cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int ragged_resident_ctas() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(kRaggedCluster * kMinBlocks * sms), 1, 1);
    cfg.blockDim = dim3((unsigned)kThreads, 1, 1);
    cfg.dynamicSmemBytes = kSmem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kRaggedCluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, ragged_kernel_fwd(), &cfg) != cudaSuccess) return 0;
    return clusters * kRaggedCluster;
}

}  // namespace sdft
