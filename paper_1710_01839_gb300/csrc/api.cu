// C-ABI entry points of libmpgemm (declared in include/mpgemm.h): argument
// checks, dispatch to the kernels, device status word, workspace.
#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "strassen.h"
#include "tc_levels.h"
#include "tune.h"

namespace mpg {

__device__ unsigned g_device_status;

static thread_local int t_last_cuda_error = 0;

void set_last_cuda_error(cudaError_t e) { t_last_cuda_error = (int)e; }

// ---------------------------------------------------------------- host fault injection
//
// One armed fault: the (after + 1)-th device allocation (FAULT_ALLOC) or
// launch check (FAULT_LAUNCH) the library makes from now on reports a
// failure, then the fault disarms.  Nothing is done to the GPU: an injected
// allocation failure allocates nothing, an injected launch failure is
// reported after a launch that did run, so the error paths that follow
// (workspace released, plan torn down) run as they would for a real one.
static std::atomic<int> g_fault_kind{0};
static std::atomic<long long> g_fault_left{0};
static std::atomic<int> g_fault_fired{0};

static void fault_from_env() {
    static std::once_flag once;
    std::call_once(once, [] {
        const char* v = getenv("MPGEMM_FAULT");
        if (!v) return;
        int kind = !strncmp(v, "alloc:", 6) ? FAULT_ALLOC : !strncmp(v, "launch:", 7) ? FAULT_LAUNCH : 0;
        if (!kind) return;
        const char* num = strchr(v, ':') + 1;
        char* end = nullptr;
        long long after = strtoll(num, &end, 10);
        if (end == num || *end || after < 0) return;
        g_fault_left.store(after);
        g_fault_kind.store(kind);
    });
}

bool fault_fire(int kind) {
    fault_from_env();
    if (g_fault_kind.load() != kind) return false;
    if (g_fault_left.fetch_sub(1) != 0) return false;
    g_fault_kind.store(0);
    g_fault_fired.fetch_add(1);
    return true;
}

cudaError_t dev_malloc(void** p, size_t bytes) {
    if (fault_fire(FAULT_ALLOC)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t s) {
    if (fault_fire(FAULT_ALLOC)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, s);
}

int check_launch() {
    if (fault_fire(FAULT_LAUNCH)) {
        set_last_cuda_error(cudaErrorLaunchFailure);
        return MPGEMM_ECUDA;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return MPGEMM_ECUDA;
    }
    return MPGEMM_OK;
}

static std::mutex g_mu;
static unsigned* g_status_ptr[64];

unsigned* device_status_ptr() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_status_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_device_status);
        if (e != cudaSuccess) {
            set_last_cuda_error(e);
            return nullptr;
        }
        g_status_ptr[dev] = static_cast<unsigned*>(p);
    }
    return g_status_ptr[dev];
}

// ---------------------------------------------------------------- workspace

static void* g_ws_ptr[64];
static size_t g_ws_bytes[64];

int workspace_get(size_t bytes, cudaStream_t s, void** out, bool* owned) {
    *out = nullptr;
    *owned = false;
    if (bytes == 0) return MPGEMM_OK;
    if (fault_fire(FAULT_ALLOC)) {   // an injected failure of the allocation below
        set_last_cuda_error(cudaErrorMemoryAllocation);
        return MPGEMM_ENOMEM;
    }
    int dev = 0;
    MPG_CUDA(cudaGetDevice(&dev));
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (dev >= 0 && dev < 64 && g_ws_ptr[dev]) {
            if (g_ws_bytes[dev] < bytes) return MPGEMM_ENOMEM;
            *out = g_ws_ptr[dev];
            return MPGEMM_OK;
        }
    }
    cudaError_t e = cudaMallocAsync(out, bytes, s);
    if (e != cudaSuccess) {
        set_last_cuda_error(e);
        return e == cudaErrorMemoryAllocation ? MPGEMM_ENOMEM : MPGEMM_ECUDA;
    }
    *owned = true;
    return MPGEMM_OK;
}

int workspace_release(void* p, bool owned, cudaStream_t s) {
    if (owned && p) MPG_CUDA(cudaFreeAsync(p, s));
    return MPGEMM_OK;
}

// ---------------------------------------------------------------- checks

static bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
    if (!a || !b || na == 0 || nb == 0) return false;
    uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + nb && y < x + na;
}

static bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int check_common(int64_t m, int64_t l, int64_t n, size_t elem_bytes, const void* A, const void* B, const void* C,
                 int algo, int n_min, int depth) {
    if (m < 0 || l < 0 || n < 0) return MPGEMM_EINVAL;
    if (m > (1LL << 31) || l > (1LL << 31) || n > (1LL << 31)) return MPGEMM_EINVAL;
    if (algo < MPGEMM_SIMPLE || algo > MPGEMM_AUTO) return MPGEMM_EINVAL;
    if (n_min > 0 && (!pow2(n_min) || n_min > 1024)) return MPGEMM_EINVAL;
    if (depth < 0 || depth > 4) return MPGEMM_EINVAL;
    size_t na = (size_t)(m * l) * elem_bytes, nb = (size_t)(l * n) * elem_bytes, nc = (size_t)(m * n) * elem_bytes;
    if ((na && !A) || (nb && !B) || (nc && !C)) return MPGEMM_EINVAL;
    if (overlaps(C, nc, A, na) || overlaps(C, nc, B, nb)) return MPGEMM_EINVAL;
    if (algo == MPGEMM_STRASSEN && depth > 0) {
        // the level-1 operand and assembly kernels put the rows of a half in grid.y
        if ((strassen_extended(m, depth) >> 1) > 65535 || (strassen_extended(l, depth) >> 1) > 65535)
            return MPGEMM_EUNSUPPORTED;
    }
    return MPGEMM_OK;
}

int default_n_min(int kind) { return kind == MPGEMM_KIND_DD ? 64 : kind == MPGEMM_KIND_QD ? 32 : 16; }

// C = 0 when l == 0 (empty sums), in every format.
template <class T>
static int zero_result(int kind, int64_t m, int64_t n, int words, T* C, cudaStream_t s) {
    size_t N = (size_t)(m * n);
    MPG_CUDA(cudaMemsetAsync(C, 0, N * (size_t)words * sizeof(T), s));
    if (kind == MPGEMM_KIND_MP) return fill_u32(reinterpret_cast<uint32_t*>(C) + N, N, 2u, s);   // flags: zero
    return MPGEMM_OK;
}

// ---------------------------------------------------------------- DD / QD

static int ddqd_entry(int kind, int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C,
                      int algo, int n_min, int depth, void* stream) {
    const int P = kind == MPGEMM_KIND_DD ? 2 : 4;
    int rc = check_common(m, l, n, sizeof(double) * P, A, B, C, algo, n_min, depth);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    PartitionScope pscope(s);
    if (m == 0 || n == 0) return MPGEMM_OK;
    if (l == 0) return zero_result<double>(kind, m, n, P, C, s);
    if (algo == MPGEMM_AUTO) {
        Choice ch;
        rc = auto_choice_measured(kind, 0, m, l, n, A, B, C, s, &ch);
        if (rc) return rc;
        algo = ch.algo;
        n_min = ch.n_min;
        depth = ch.depth;
    }
    if (n_min <= 0) n_min = default_n_min(kind);
    const size_t eb = sizeof(double) * P;
    View<const double> a = bounded(planes_view(A, m, l), A, eb * m * l);
    View<const double> b = bounded(planes_view(B, l, n), B, eb * l * n);
    View<double> c = bounded(planes_view(C, m, n), C, eb * m * n);
    if (algo == MPGEMM_STRASSEN && depth > 0) return strassen_ddqd(kind, m, l, n, a, b, c, n_min, depth, s);
    return ddqd_gemm(kind, algo == MPGEMM_SIMPLE ? MPGEMM_SIMPLE : MPGEMM_BLOCK, m, l, n, 1, a, b, c, n_min, s);
}

static int mp_entry(int64_t m, int64_t l, int64_t n, int prec_bits, const uint32_t* A, const uint32_t* B,
                    uint32_t* C, int algo, int n_min, int depth, void* stream) {
    if (prec_bits <= 0 || prec_bits % 32) return MPGEMM_EINVAL;
    int w = prec_bits / 32;
    if (!(w == 1 || w == 2 || w == 4 || w == 8 || w == 16 || w == 32 || w == 64)) return MPGEMM_EUNSUPPORTED;
    int rc = check_common(m, l, n, sizeof(uint32_t) * (size_t)(2 + w), A, B, C, algo, n_min, depth);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    PartitionScope pscope(s);
    if (m == 0 || n == 0) return MPGEMM_OK;
    if (l == 0) return zero_result<uint32_t>(MPGEMM_KIND_MP, m, n, 2 + w, C, s);
    if (algo == MPGEMM_AUTO) {
        Choice ch;
        rc = auto_choice_measured(MPGEMM_KIND_MP, prec_bits, m, l, n, A, B, C, s, &ch);
        if (rc) return rc;
        algo = ch.algo;
        n_min = ch.n_min;
        depth = ch.depth;
    }
    if (n_min <= 0) n_min = default_n_min(MPGEMM_KIND_MP);
    const size_t eb = sizeof(uint32_t) * (size_t)(2 + w);
    View<const uint32_t> a = bounded(planes_view(A, m, l), A, eb * m * l);
    View<const uint32_t> b = bounded(planes_view(B, l, n), B, eb * l * n);
    View<uint32_t> c = bounded(planes_view(C, m, n), C, eb * m * n);
    if (algo == MPGEMM_STRASSEN && depth > 0) return strassen_mp(w, m, l, n, a, b, c, n_min, depth, s);
    return mp_gemm(w, algo == MPGEMM_SIMPLE ? MPGEMM_SIMPLE : MPGEMM_BLOCK, m, l, n, 1, a, b, c, n_min, s);
}

#ifdef MPGEMM_BOUNDS_CHECK
BoundsWord* bounds_word() {
    static BoundsWord* words[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!words[dev]) {
        void* p = nullptr;
        if (cudaMalloc(&p, sizeof(BoundsWord)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(BoundsWord)) != cudaSuccess) return nullptr;
        words[dev] = static_cast<BoundsWord*>(p);
    }
    return words[dev];
}

// One thread reads element 3 of a 16-word buffer (inside), then element 16
// and writes element -1 (both outside: not made, counted).
__global__ void k_selftest_bounds(View<uint32_t> V, uint32_t* out) {
    out[0] = V.load(V.at(0, 0, 0, 3));
    out[1] = V.load(V.at(0, 0, 0, 16));
    V.store(V.at(0, 0, 0, -1), 7u);
}

static int bounds_selftest(cudaStream_t s) {
    static uint32_t* buf = nullptr;
    if (!buf) {
        void* p = nullptr;
        MPG_CUDA(cudaMalloc(&p, 32 * sizeof(uint32_t)));
        MPG_CUDA(cudaMemset(p, 0, 32 * sizeof(uint32_t)));
        buf = static_cast<uint32_t*>(p);
    }
    // the view covers words 8 .. 23 of the allocation: the probes outside it
    // stay inside the allocation, whether or not the check works
    View<uint32_t> v = bounded(planes_view(buf + 8, 1, 16), buf + 8, 16 * sizeof(uint32_t));
    k_selftest_bounds<<<1, 1, 0, s>>>(v, buf + 28);
    return check_launch();
}
#endif

}  // namespace mpg

using namespace mpg;

extern "C" {

int mpgemm_dd(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int algo, int n_min,
              int strassen_depth, void* stream) {
    return ddqd_entry(MPGEMM_KIND_DD, m, l, n, A, B, C, algo, n_min, strassen_depth, stream);
}

int mpgemm_qd(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int algo, int n_min,
              int strassen_depth, void* stream) {
    return ddqd_entry(MPGEMM_KIND_QD, m, l, n, A, B, C, algo, n_min, strassen_depth, stream);
}

int mpgemm_mp(int64_t m, int64_t l, int64_t n, int prec_bits, const uint32_t* A, const uint32_t* B, uint32_t* C,
              int algo, int n_min, int strassen_depth, void* stream) {
    return mp_entry(m, l, n, prec_bits, A, B, C, algo, n_min, strassen_depth, stream);
}

size_t mpgemm_workspace_size(int kind, int prec_bits, int64_t m, int64_t l, int64_t n, int algo,
                             int strassen_depth) {
    if (algo != MPGEMM_STRASSEN || strassen_depth <= 0 || m <= 0 || l <= 0 || n <= 0) return 0;
    size_t eb;
    if (kind == MPGEMM_KIND_DD) eb = 2 * sizeof(double);
    else if (kind == MPGEMM_KIND_QD) eb = 4 * sizeof(double);
    else if (kind == MPGEMM_KIND_MP && prec_bits > 0 && prec_bits % 32 == 0) eb = sizeof(uint32_t) * (size_t)(2 + prec_bits / 32);
    else return 0;
    return strassen_workspace_bytes(eb, m, l, n, strassen_depth);
}

int mpgemm_set_workspace(void* dev_ptr, size_t bytes) {
    int dev = 0;
    MPG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return MPGEMM_EINVAL;
    if ((dev_ptr == nullptr) != (bytes == 0)) return MPGEMM_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    g_ws_ptr[dev] = dev_ptr;
    g_ws_bytes[dev] = bytes;
    return MPGEMM_OK;
}

int mpgemm_stream_status(void* stream) {
    PartitionScope pscope((cudaStream_t)stream);
    MPG_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned* p = device_status_ptr();
    if (!p) return MPGEMM_ECUDA;
    unsigned v = 0;
    MPG_CUDA(cudaMemcpy(&v, p, sizeof v, cudaMemcpyDeviceToHost));
    if (v) {
        unsigned zero = 0;
        MPG_CUDA(cudaMemcpy(p, &zero, sizeof zero, cudaMemcpyHostToDevice));
    }
    if (v & DEV_EXP_OVERFLOW) return MPGEMM_EOVERFLOW;
    if (v & DEV_TIMEOUT) return MPGEMM_ETIMEOUT;
    if (v & (DEV_BAD_DESC | DEV_NONFINITE)) return MPGEMM_EINVAL;
    return MPGEMM_OK;
}

const char* mpgemm_strerror(int status) {
    switch (status) {
        case MPGEMM_OK: return "ok";
        case MPGEMM_EINVAL: return "invalid argument";
        case MPGEMM_EUNSUPPORTED: return "unsupported configuration";
        case MPGEMM_ECUDA: return "CUDA error";
        case MPGEMM_EOVERFLOW: return "multi-limb exponent overflow";
        case MPGEMM_ETIMEOUT: return "device wait timed out";
        case MPGEMM_ENOMEM: return "out of device memory or workspace too small";
        default: return "unknown status";
    }
}

int mpgemm_last_cuda_error(void) { return t_last_cuda_error; }

int mpgemm_fault_inject(int what, long long after) {
    fault_from_env();   // an environment setting read later would override this call
    if (what < 0 || what > FAULT_LAUNCH || after < 0) return MPGEMM_EINVAL;
    g_fault_kind.store(0);
    g_fault_left.store(after);
    g_fault_kind.store(what);
    return MPGEMM_OK;
}

int mpgemm_fault_fired(void) { return g_fault_fired.load(); }

int mpgemm_selftest_wait_timeout(int limit_ms, void* stream) {
    cudaStream_t s = (cudaStream_t)stream;
    PartitionScope pscope(s);
    int rc = wait_selftest(limit_ms, s);
    if (rc) return rc;
    return mpgemm_stream_status(stream);
}

int mpgemm_version(void) { return 10000 * 0 + 100 * 2 + 0; }

int mpgemm_bounds_read(long long* count, unsigned long long* first_address) {
#ifdef MPGEMM_BOUNDS_CHECK
    if (!count || !first_address) return MPGEMM_EINVAL;
    BoundsWord* w = bounds_word();
    if (!w) return MPGEMM_ECUDA;
    BoundsWord h{};
    MPG_CUDA(cudaDeviceSynchronize());
    MPG_CUDA(cudaMemcpy(&h, w, sizeof h, cudaMemcpyDeviceToHost));
    MPG_CUDA(cudaMemset(w, 0, sizeof h));
    *count = (long long)h.count;
    *first_address = h.first;
    return MPGEMM_OK;
#else
    (void)count;
    (void)first_address;
    return MPGEMM_EUNSUPPORTED;
#endif
}

int mpgemm_selftest_bounds(void* stream) {
#ifdef MPGEMM_BOUNDS_CHECK
    return bounds_selftest((cudaStream_t)stream);
#else
    (void)stream;
    return MPGEMM_EUNSUPPORTED;
#endif
}

}  // extern "C"
