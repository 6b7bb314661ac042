// SM partitions: streams whose kernels run on a subset of the SMs (CUDA
// green contexts).  They are the GPU counterpart of the paper's thread-count
// axis (Section 4 times every algorithm with 1, 2, 4 and 8 OpenMP threads):
// the same library calls, issued on a partition's stream, run on that many
// SMs, and the parts of the library that size work by the SM count (the
// tuner's rounds model and remembered choices, the cost model's features,
// the persistent tcgen05 kernel's grid) read the partition's count through
// stream_sms().
//
// The driver functions are resolved through the runtime's driver entry
// point, so the library does not link against the driver library.  A green
// context only restricts where this process's kernels run; it changes no
// device setting.
#include <cuda.h>

#include <map>
#include <mutex>

#include "common.cuh"

namespace mpg {

namespace {

struct GreenFns {
    CUresult (*device_get)(CUdevice*, int) = nullptr;
    CUresult (*device_resource)(CUdevice, CUdevResource*, CUdevResourceType) = nullptr;
    CUresult (*split)(CUdevResource*, unsigned*, const CUdevResource*, CUdevResource*, unsigned, unsigned) = nullptr;
    CUresult (*make_desc)(CUdevResourceDesc*, CUdevResource*, unsigned) = nullptr;
    CUresult (*ctx_create)(CUgreenCtx*, CUdevResourceDesc, CUdevice, unsigned) = nullptr;
    CUresult (*ctx_destroy)(CUgreenCtx) = nullptr;
    CUresult (*stream_create)(CUstream*, CUgreenCtx, unsigned, int) = nullptr;
    CUresult (*stream_destroy)(CUstream) = nullptr;
    CUresult (*to_ctx)(CUcontext*, CUgreenCtx) = nullptr;
    CUresult (*push)(CUcontext) = nullptr;
    CUresult (*pop)(CUcontext*) = nullptr;
    bool ok = false;
};

template <class F>
static bool resolve(const char* name, unsigned version, F& fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
        return false;
    fn = reinterpret_cast<F>(p);
    return true;
}

static const GreenFns& green() {
    static GreenFns g;
    static std::once_flag once;
    std::call_once(once, [] {
        g.ok = resolve("cuDeviceGet", 12000, g.device_get) &&
               resolve("cuDeviceGetDevResource", 12040, g.device_resource) &&
               resolve("cuDevSmResourceSplitByCount", 12040, g.split) &&
               resolve("cuDevResourceGenerateDesc", 12040, g.make_desc) &&
               resolve("cuGreenCtxCreate", 12040, g.ctx_create) &&
               resolve("cuGreenCtxDestroy", 12040, g.ctx_destroy) &&
               resolve("cuGreenCtxStreamCreate", 12050, g.stream_create) &&
               resolve("cuStreamDestroy", 12000, g.stream_destroy) &&
               resolve("cuCtxFromGreenCtx", 12040, g.to_ctx) && resolve("cuCtxPushCurrent", 12000, g.push) &&
               resolve("cuCtxPopCurrent", 12000, g.pop);
    });
    return g;
}

struct Partition {
    CUgreenCtx green;
    CUcontext ctx;   // the green context as a context the runtime can use
    int sms;
};

std::mutex g_pmu;
std::map<cudaStream_t, Partition> g_parts;

int device_sms() {
    static int sms[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 152;
    return sms[dev];
}

}  // namespace

// The runtime issues work into the context current on the calling thread,
// so a call on a partition's stream makes the partition's context current
// for its duration.
// Addresses of the library's __device__ words are resolved (and cached per
// device) in the context that was current before the push, the device's
// primary context: a green context's own module copy would go away with the
// partition, and a cached address of it would then dangle.
PartitionScope::PartitionScope(cudaStream_t s) {
    CUcontext c = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_pmu);
        auto it = g_parts.find(s);
        if (it == g_parts.end()) return;
        c = it->second.ctx;
    }
    (void)device_status_ptr();
    pushed_ = green().push(c) == CUDA_SUCCESS;
}

PartitionScope::~PartitionScope() {
    if (pushed_) {
        CUcontext c;
        green().pop(&c);
    }
}

int stream_sms(cudaStream_t s) {
    {
        std::lock_guard<std::mutex> lk(g_pmu);
        auto it = g_parts.find(s);
        if (it != g_parts.end()) return it->second.sms;
    }
    return device_sms();
}

}  // namespace mpg

using namespace mpg;

extern "C" {

int mpgemm_partition_create(int num_sms, void** stream, int* sms_out) {
    if (!stream || num_sms <= 0) return MPGEMM_EINVAL;
    *stream = nullptr;
    const GreenFns& g = green();
    if (!g.ok) return MPGEMM_EUNSUPPORTED;
    int dev = 0;
    MPG_CUDA(cudaGetDevice(&dev));
    MPG_CUDA(cudaFree(nullptr));   // the primary context is current before green contexts are made
    CUdevice cd;
    if (g.device_get(&cd, dev) != CUDA_SUCCESS) return MPGEMM_ECUDA;
    CUdevResource all;
    if (g.device_resource(cd, &all, CU_DEV_RESOURCE_TYPE_SM) != CUDA_SUCCESS) return MPGEMM_ECUDA;
    if ((unsigned)num_sms > all.sm.smCount) return MPGEMM_EINVAL;
    CUdevResource part;
    unsigned groups = 1;
    if (g.split(&part, &groups, &all, nullptr, 0, (unsigned)num_sms) != CUDA_SUCCESS || groups < 1)
        return MPGEMM_EUNSUPPORTED;
    CUdevResourceDesc desc;
    if (g.make_desc(&desc, &part, 1) != CUDA_SUCCESS) return MPGEMM_ECUDA;
    CUgreenCtx ctx;
    if (g.ctx_create(&ctx, desc, cd, CU_GREEN_CTX_DEFAULT_STREAM) != CUDA_SUCCESS) return MPGEMM_ECUDA;
    CUcontext cc;
    CUstream cs;
    if (g.to_ctx(&cc, ctx) != CUDA_SUCCESS || g.stream_create(&cs, ctx, CU_STREAM_NON_BLOCKING, 0) != CUDA_SUCCESS) {
        g.ctx_destroy(ctx);
        return MPGEMM_ECUDA;
    }
    {
        std::lock_guard<std::mutex> lk(g_pmu);
        g_parts[(cudaStream_t)cs] = Partition{ctx, cc, (int)part.sm.smCount};
    }
    *stream = (void*)cs;
    if (sms_out) *sms_out = (int)part.sm.smCount;
    return MPGEMM_OK;
}

int mpgemm_partition_destroy(void* stream) {
    Partition p;
    {
        std::lock_guard<std::mutex> lk(g_pmu);
        auto it = g_parts.find((cudaStream_t)stream);
        if (it == g_parts.end()) return MPGEMM_EINVAL;
        p = it->second;
        g_parts.erase(it);
    }
    const GreenFns& g = green();
    int rc = MPGEMM_OK;
    if (g.push(p.ctx) == CUDA_SUCCESS) {
        if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) rc = MPGEMM_ECUDA;
        CUcontext c;
        g.pop(&c);
    }
    if (g.stream_destroy((CUstream)stream) != CUDA_SUCCESS) rc = MPGEMM_ECUDA;
    if (g.ctx_destroy(p.green) != CUDA_SUCCESS) rc = MPGEMM_ECUDA;
    return rc;
}

int mpgemm_stream_sms(void* stream) { return stream_sms((cudaStream_t)stream); }

}  // extern "C"
