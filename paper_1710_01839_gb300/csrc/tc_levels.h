// tcgen05 level-sum kernel of the FP8-digit split-precision DD GEMM.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mpg {

// L_g (S int32 planes of m x n) from e4m3 digit planes (S planes of m x lp and
// n x lp, K contiguous, lp a multiple of 128).  Requires 256 * lp <= 2^24.
int tc_levels(int64_t m, int64_t n, int64_t lp, int S, const void* DA, const void* DB, int* Lv, cudaStream_t s);

// Launches the bounded-wait self-test (a wait nothing completes, limit_ms
// 1..2000); the status word then reads DEV_TIMEOUT.
int wait_selftest(int limit_ms, cudaStream_t s);

}  // namespace mpg
