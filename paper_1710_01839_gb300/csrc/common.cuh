// Shared definitions of the multiple-precision GEMM library (device side).
//
// Matrix storage: row-major "planes".  A DD matrix is two contiguous arrays
// [hi | lo] of rows*cols doubles, QD four planes, a p-bit multi-limb matrix
// (2 + w) planes of uint32 words [exponent | flags | limb 0 .. limb w-1].
// Internally every operand is addressed through a View: element (z, q, i, j)
// (batch z, plane q, row i, column j) lives at p[z*bs + q*ps + i*ld + j], so
// Strassen's quadrants and batched sub-problems need no copies.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/mpgemm.h"

namespace mpg {

#ifdef MPGEMM_BOUNDS_CHECK
// The bounds-checked build (-DMPGEMM_BOUNDS_CHECK, libmpgemm_bc.so): a view
// also knows the buffer it addresses, [lo, hi), and the GEMM kernels read
// and write global memory only through View::load / get / store, which
// check the element against it.  An element outside is not accessed (a load
// reads 0); the miss is counted in `oob` and the first missed address kept,
// for mpgemm_bounds_read().  A view without a buffer (lo null) is unchecked.
struct BoundsWord {
    unsigned long long count;
    unsigned long long first;
};
BoundsWord* bounds_word();   // this device's counter (device memory)
#endif

template <class T>
struct View {
    T* p;
    int64_t ld;  // row stride (elements)
    int64_t ps;  // plane stride (elements)
    int64_t bs;  // batch stride (elements)
#ifdef MPGEMM_BOUNDS_CHECK
    const void* lo = nullptr;
    const void* hi = nullptr;
    BoundsWord* oob = nullptr;
#endif
    __host__ __device__ T* at(int64_t z, int q, int64_t i, int64_t j) const {
        return p + z * bs + q * ps + i * ld + j;
    }
    // whether element q may be accessed (always, outside the checked build)
    __device__ __forceinline__ bool ok(const T* q) const {
#ifdef MPGEMM_BOUNDS_CHECK
        if (lo && ((const char*)q < (const char*)lo || (const char*)(q + 1) > (const char*)hi)) {
            if (atomicAdd(&oob->count, 1ull) == 0ull) oob->first = (unsigned long long)(uintptr_t)q;
            return false;
        }
#endif
        return true;
    }
    // read-only load through the non-coherent cache (operands)
    __device__ __forceinline__ T load(const T* q) const { return ok(q) ? __ldg(q) : T(0); }
    // plain load (workspace the same kernel sequence writes)
    __device__ __forceinline__ T get(const T* q) const { return ok(q) ? *q : T(0); }
    __device__ __forceinline__ void store(T* q, T v) const {
        if (ok(q)) *q = v;
    }
};

template <class T>
__host__ __device__ inline View<T> planes_view(T* p, int64_t rows, int64_t cols) {
    View<T> v{p, cols, rows * cols, 0};
    return v;
}

// v restricted to the buffer [base, base + bytes) in the checked build (the
// view itself elsewhere).
template <class T>
inline View<T> bounded(View<T> v, const void* base, size_t bytes) {
#ifdef MPGEMM_BOUNDS_CHECK
    v.oob = bounds_word();
    if (v.oob) {   // no counter (allocation failed): the view stays unchecked
        v.lo = base;
        v.hi = (const char*)base + bytes;
    }
#else
    (void)base;
    (void)bytes;
#endif
    return v;
}

// Device-side status word (bits of MPGEMM_DEV_*), one per device, read and
// cleared by mpgemm_stream_status().
enum : unsigned {
    DEV_EXP_OVERFLOW = 1u,   // a multi-limb exponent left the int32 range (or a
                             // conversion to double left the normal range)
    DEV_TIMEOUT = 2u,        // a bounded wait in a persistent kernel gave up
    DEV_BAD_DESC = 4u,       // a batched descriptor failed a device-side check
    DEV_NONFINITE = 8u,      // a conversion to multi-limb met an infinity or NaN
};

unsigned* device_status_ptr();   // address of this device's status word
int stream_sms(cudaStream_t s);   // SMs the stream's kernels run on (an SM partition's, else the device's)
// Makes an SM partition's context current while a call issues work on the
// partition's stream (no-op for other streams).
class PartitionScope {
   public:
    explicit PartitionScope(cudaStream_t s);
    ~PartitionScope();
    PartitionScope(const PartitionScope&) = delete;
    PartitionScope& operator=(const PartitionScope&) = delete;

   private:
    bool pushed_ = false;
};

// Launch-shape helpers.
__host__ __device__ inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Host-side error plumbing.
#define MPG_CUDA(call)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) {                              \
            ::mpg::set_last_cuda_error(e_);                   \
            return MPGEMM_ECUDA;                              \
        }                                                     \
    } while (0)

void set_last_cuda_error(cudaError_t e);
int check_launch();   // cudaGetLastError -> status (or an injected launch failure)

// Host fault injection (mpgemm_fault_inject, MPGEMM_FAULT): true when the
// armed fault of this kind fires now.  Device allocations of the library go
// through dev_malloc / dev_malloc_async (or workspace_get), which honour it.
enum { FAULT_ALLOC = 1, FAULT_LAUNCH = 2 };
bool fault_fire(int kind);
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t s);

// CTA raster order: with group size G (in tiles), consecutive CTA ids cover a
// G x G super-tile of C before moving on (G = 1 is plain row-major order).
__device__ __forceinline__ void raster(unsigned pid, unsigned tiles_m, unsigned tiles_n, unsigned G,
                                       unsigned& tm, unsigned& tn) {
    unsigned band = G * tiles_n;
    unsigned gid = pid / band;
    unsigned first = gid * G;
    unsigned gm = tiles_m - first < G ? tiles_m - first : G;
    unsigned r = pid - gid * band;
    tm = first + r % gm;
    tn = r / gm;
}

}  // namespace mpg
