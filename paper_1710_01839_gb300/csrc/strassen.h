// Strassen's algorithm (Eq 3) on the GPU, breadth first: each recursion
// level forms the operands of all 7^k sub-products in one batched
// elementwise launch, all 7^d leaf products run as ONE batched block-GEMM
// launch, and the C quadrants are assembled level by level in one batched
// launch each.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace mpg {

// x rounded up to a multiple of 2^depth: Strassen's zero-extended size.
int64_t strassen_extended(int64_t x, int depth);
// Workspace of Strassen at the zero-extended sizes.
size_t strassen_workspace_bytes(size_t elem_bytes, int64_t m, int64_t l, int64_t n, int depth);

int strassen_ddqd(int kind, int64_t m, int64_t l, int64_t n, View<const double> A, View<const double> B,
                  View<double> C, int n_min, int depth, cudaStream_t s);
int strassen_mp(int w, int64_t m, int64_t l, int64_t n, View<const uint32_t> A, View<const uint32_t> B,
                View<uint32_t> C, int n_min, int depth, cudaStream_t s);

// Strassen with caller-provided workspace (ws, ws_bytes >= the size above).
int strassen_ddqd_ws(int kind, int64_t m, int64_t l, int64_t n, View<const double> A, View<const double> B,
                     View<double> C, int n_min, int depth, void* ws, size_t ws_bytes, cudaStream_t s);
int strassen_mp_ws(int w, int64_t m, int64_t l, int64_t n, View<const uint32_t> A, View<const uint32_t> B,
                   View<uint32_t> C, int n_min, int depth, void* ws, size_t ws_bytes, cudaStream_t s);

int fill_u32(uint32_t* p, size_t count, uint32_t value, cudaStream_t s);

// Workspace plumbing shared by the entry points (api.cu).
int workspace_get(size_t bytes, cudaStream_t s, void** out, bool* owned);
int workspace_release(void* p, bool owned, cudaStream_t s);

}  // namespace mpg
