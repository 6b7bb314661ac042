// Internal launch interfaces between the C-ABI layer and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace mpg {

// DD / QD simple (Eq 1) or block (Eq 2) over `batch` independent problems
// (grid.z / grid.y); kind = MPGEMM_KIND_DD or MPGEMM_KIND_QD.
int ddqd_gemm(int kind, int algo, int64_t m, int64_t l, int64_t n, int64_t batch, View<const double> A,
              View<const double> B, View<double> C, int n_min, cudaStream_t s);

// While alive, multi-limb GEMMs issued from this host thread expect
// operands of similar magnitude (the integer pipe's images of DD / QD
// numbers) and use the add's alignment shortcut for them.
class CloseOperandsScope {
   public:
    CloseOperandsScope();
    ~CloseOperandsScope();
    CloseOperandsScope(const CloseOperandsScope&) = delete;
    CloseOperandsScope& operator=(const CloseOperandsScope&) = delete;

   private:
    bool prev_;
};

// Multi-limb simple / block, w limbs per mantissa.
int mp_gemm(int w, int algo, int64_t m, int64_t l, int64_t n, int64_t batch, View<const uint32_t> A,
            View<const uint32_t> B, View<uint32_t> C, int n_min, cudaStream_t s);

// Multi-limb block GEMM with a team of w / 8 lanes per output (w = 16, 32,
// 64); mp_team_leaf says whether mp_gemm's block algorithm uses it for a
// batch of m x n outputs on stream s.
bool mp_team_leaf(int w, int64_t m, int64_t n, int64_t batch, cudaStream_t s);
int mp_gemm_team(int w, int64_t m, int64_t l, int64_t n, int64_t batch, View<const uint32_t> A,
                 View<const uint32_t> B, View<uint32_t> C, int n_min, unsigned* status, cudaStream_t s);

// Elementwise z = x + y (sub: x - y) in a format over a batch of r x c matrices.
int ddqd_addsub(int kind, int64_t r, int64_t c, int64_t batch, View<double> Z, View<const double> X,
                View<const double> Y, int sub, cudaStream_t s);
int mp_addsub(int w, int64_t r, int64_t c, int64_t batch, View<uint32_t> Z, View<const uint32_t> X,
              View<const uint32_t> Y, int sub, cudaStream_t s);

// Host-checkable argument errors of a GEMM call (sizes, algo, n_min, depth,
// null or overlapping buffers of elem_bytes per element); MPGEMM_OK if none.
int check_common(int64_t m, int64_t l, int64_t n, size_t elem_bytes, const void* A, const void* B, const void* C,
                 int algo, int n_min, int depth);

}  // namespace mpg
