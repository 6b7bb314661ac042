// Split-precision DD GEMM (Ozaki-style): internal interfaces.  kind 0 = int8
// base-128 digits, kind 1 = FP8 e4m3 balanced base-32 digits.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace mpg {

int64_t ozaki_padded_k(int64_t l);
size_t ozaki_workspace_bytes(int64_t m, int64_t l, int64_t n, int S);
int ozaki_split(int kind, int by_col, int64_t rows, int64_t cols, const double* X, int S, int* expo, void* D,
                int64_t lp, cudaStream_t s);
int ozaki_levels(int kind, int64_t m, int64_t n, int64_t lp, int S, const void* DA, const void* DB, int* Lv,
                 cudaStream_t s);
int ozaki_recombine(int kind, int64_t m, int64_t n, int S, const int* Lv, const int* e, const int* f, double* C,
                    cudaStream_t s);
int ozaki_gemm_ws(int kind, int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int S,
                  void* ws, size_t ws_bytes, cudaStream_t s);

}  // namespace mpg
