// DD Strassen with library-owned scratch: for callers that must not allocate
// device memory while they run.
//
// The regular entry point (mpgemm_dd with MPGEMM_STRASSEN) takes its
// workspace from mpgemm_set_workspace or allocates it per call with
// cudaMallocAsync.  Some callers can do neither: a service that hands all of
// a GPU's memory to its own pool allocator at start-up and forbids any other
// allocation afterwards, or a latency-critical loop in which an allocation's
// possible device-wide synchronisation or failure is not acceptable.  This
// variant runs the same kernels on a fixed scratch array that lives in the
// library's own device memory (a file-scope __device__ array), so it never
// allocates.
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "strassen.h"
#include "tune.h"

namespace mpg {

// Scratch for the Strassen operands and products.  Every GPU that loads the
// library holds these bytes until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

static std::mutex g_na_mu;
static void* g_na_ptr[64];

// Device address of the scratch array for the current device.  In host code
// the array's name is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress, once per device with that device current.  It
// is resolved before a partition's (green) context is pushed, so the cached
// address is the primary context's array, which every partition of the
// device can use and which outlives any partition.
static int noalloc_scratch(void** out) {
    int dev = 0;
    MPG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return MPGEMM_EUNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        MPG_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_na_ptr[dev] = p;
    }
    *out = g_na_ptr[dev];
    return MPGEMM_OK;
}

}  // namespace mpg

using namespace mpg;

extern "C" {

int mpgemm_dd_strassen_noalloc(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C,
                               int n_min, int strassen_depth, void* stream) {
    if (strassen_depth < 1) return MPGEMM_EINVAL;
    int rc = check_common(m, l, n, 2 * sizeof(double), A, B, C, MPGEMM_STRASSEN, n_min, strassen_depth);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (m == 0 || n == 0) return MPGEMM_OK;
    if (l == 0) {   // empty sums: C = 0
        PartitionScope pscope(s);
        MPG_CUDA(cudaMemsetAsync(C, 0, 2 * sizeof(double) * (size_t)(m * n), s));
        return MPGEMM_OK;
    }
    const size_t bytes = strassen_workspace_bytes(2 * sizeof(double), m, l, n, strassen_depth);
    if (bytes > NOALLOC_SCRATCH_BYTES) return MPGEMM_ENOMEM;   // problem too large for the fixed scratch
    void* ws = nullptr;
    if ((rc = noalloc_scratch(&ws))) return rc;
    PartitionScope pscope(s);   // a partition's stream: its kernels run in its context
    if (n_min <= 0) n_min = default_n_min(MPGEMM_KIND_DD);
    const size_t eb = 2 * sizeof(double);
    View<const double> a = bounded(planes_view(A, m, l), A, eb * m * l);
    View<const double> b = bounded(planes_view(B, l, n), B, eb * l * n);
    View<double> c = bounded(planes_view(C, m, n), C, eb * m * n);
    return strassen_ddqd_ws(MPGEMM_KIND_DD, m, l, n, a, b, c, n_min, strassen_depth, ws, bytes, s);
}

}  // extern "C"
