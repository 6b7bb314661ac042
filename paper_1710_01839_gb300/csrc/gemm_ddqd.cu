// DD and QD GEMM kernels: the simple algorithm (Eq 1) and the block
// algorithm (Eq 2).
//
// Both formats are FP64-pipe bound on GB300 (about 0.6 T FP64 ops/s against
// ~7 TB/s of HBM: a DD multiply-accumulate costs 12 FP64 operations for 32
// bytes of operands that are reused BM times from shared memory), so the
// design goal is to keep the FP64 pipe busy: many independent accumulators
// per thread, operands from shared memory as 16-byte (hi, lo) pairs, no FP64
// in address arithmetic, and global loads for the next K panel issued before
// the current panel's arithmetic.
#include "common.cuh"
#include "ddqd.cuh"
#include "tiles.cuh"
#include "kernels.h"
#include "profile.h"

namespace mpg {

// ---------------------------------------------------------------- Eq 1

// One thread per c_ij; k ascending; operands straight from global memory.
template <class Fmt>
__global__ void __launch_bounds__(256) k_simple(int64_t m, int64_t l, int64_t n, View<const double> A,
                                                View<const double> B, View<double> C) {
    constexpr int P = Fmt::P;
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    int64_t z = blockIdx.z;
    if (i >= m || j >= n) return;
    typename Fmt::Acc acc;
    Fmt::zero(acc);
    const double* pa = A.at(z, 0, i, 0);
    const double* pb = B.at(z, 0, 0, j);
    for (int64_t k = 0; k < l; k++) {
        double a[P], b[P];
#pragma unroll
        for (int q = 0; q < P; q++) {
            a[q] = A.load(pa + q * A.ps + k);
            b[q] = B.load(pb + q * B.ps + k * B.ld);
        }
        Fmt::mac(acc, a, b);
        if ((k + 1) % Fmt::R == 0) Fmt::renorm(acc);
    }
    double out[P];
    Fmt::finish(acc, out);
#pragma unroll
    for (int q = 0; q < P; q++) C.store(C.at(z, q, i, j), out[q]);
}

// ---------------------------------------------------------------- Eq 2

// One CTA computes a BM x BM block of C (ddqd_block_tile); CTA order follows
// the super-tile raster with group G (n_min / BM when n_min > BM).
template <class Fmt, int BM, int RM, int KT>
__global__ void __launch_bounds__((BM / RM) * (BM / RM)) k_block(int64_t m, int64_t l, int64_t n,
                                                                 View<const double> A, View<const double> B,
                                                                 View<double> C, unsigned G) {
    __shared__ __align__(16) double sm[ddqd_tile_doubles<Fmt, BM, KT>()];
    const unsigned tiles_m = ceil_div(m, BM), tiles_n = ceil_div(n, BM);
    unsigned tm, tn;
    raster(blockIdx.x, tiles_m, tiles_n, G, tm, tn);
    ddqd_block_tile<Fmt, BM, RM, KT>(m, l, n, A, B, C, blockIdx.y, (int64_t)tm * BM, (int64_t)tn * BM, sm);
}

// ---------------------------------------------------------------- launchers

template <class Fmt>
static int launch_simple(int64_t m, int64_t l, int64_t n, int64_t batch, View<const double> A,
                         View<const double> B, View<double> C, cudaStream_t s) {
    dim3 blk(32, 8);
    dim3 grd(ceil_div(n, 32), ceil_div(m, 8), (unsigned)batch);
    ProfScope ps(s);
    k_simple<Fmt><<<grd, blk, 0, s>>>(m, l, n, A, B, C);
    return check_launch();
}

template <class Fmt, int BM, int RM, int KT>
static int launch_block_cfg(int64_t m, int64_t l, int64_t n, int64_t batch, View<const double> A,
                            View<const double> B, View<double> C, int n_min, cudaStream_t s) {
    unsigned G = n_min > BM ? (unsigned)(n_min / BM) : 1u;
    constexpr int NT = (BM / RM) * (BM / RM);
    dim3 grd(ceil_div(m, BM) * ceil_div(n, BM), (unsigned)batch);
    ProfScope ps(s);
    k_block<Fmt, BM, RM, KT><<<grd, NT, 0, s>>>(m, l, n, A, B, C, G);
    return check_launch();
}

int ddqd_gemm(int kind, int algo, int64_t m, int64_t l, int64_t n, int64_t batch, View<const double> A,
              View<const double> B, View<double> C, int n_min, cudaStream_t s) {
    if (m == 0 || n == 0 || batch == 0) return MPGEMM_OK;
    if (kind == MPGEMM_KIND_DD) {
        if (algo == MPGEMM_SIMPLE) return launch_simple<DDFmt>(m, l, n, batch, A, B, C, s);
        if (n_min <= 16) return launch_block_cfg<DDFmt, 16, 1, 16>(m, l, n, batch, A, B, C, n_min, s);
        if (n_min <= 32) return launch_block_cfg<DDFmt, 32, 2, 16>(m, l, n, batch, A, B, C, n_min, s);
        return launch_block_cfg<DDFmt, 64, 4, 16>(m, l, n, batch, A, B, C, n_min, s);
    }
    if (algo == MPGEMM_SIMPLE) return launch_simple<QDFmt>(m, l, n, batch, A, B, C, s);
    if (n_min <= 16) return launch_block_cfg<QDFmt, 16, 1, 16>(m, l, n, batch, A, B, C, n_min, s);
    return launch_block_cfg<QDFmt, 32, 2, 8>(m, l, n, batch, A, B, C, n_min, s);
}

// TwoSum with the integer-pipe error term against the FP64 formula, element
// by element (mpgemm_selftest_two_sum).
__global__ void k_selftest_two_sum(int64_t count, const double* a, const double* b, double* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double s, e, s2, e2;
    two_sum(a[i], b[i], s, e);
    two_sum_fp64(a[i], b[i], s2, e2);
    out[i] = s;
    out[count + i] = e;
    out[2 * count + i] = e2;
}

// The DD MAC's product and its error on the integer pipe, with the FP64
// error fma(a, b, -RN(a b)) beside them (mpgemm_selftest_two_prod).
__global__ void k_selftest_two_prod(int64_t count, const double* a, const double* b, double* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double p, e;
    two_prod(a[i], b[i], p, e);
    out[i] = p;
    out[count + i] = e;
    out[2 * count + i] = __fma_rn(a[i], b[i], -__dmul_rn(a[i], b[i]));
}

// The DD MAC (TwoProd and TwoSum's error on the integer pipe) and its
// all-FP64 form on the same steps (mpgemm_selftest_dd_mac): in = [s, t,
// ah, al, bh, bl] planes, out = [s, t] of dd_mac then of dd_mac_fp64, then
// [s, t] after one more renormalisation (dd_renorm and two_sum_fp64).
__global__ void k_selftest_dd_mac(int64_t count, const double* in, double* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double* v = in + i;
    DDAcc c{v[0], v[count]}, f{v[0], v[count]};
    dd_mac(c, v[2 * count], v[3 * count], v[4 * count], v[5 * count]);
    dd_mac_fp64(f, v[2 * count], v[3 * count], v[4 * count], v[5 * count]);
    out[i] = c.s;
    out[count + i] = c.t;
    out[2 * count + i] = f.s;
    out[3 * count + i] = f.t;
    dd_renorm(c);
    double s, t;
    two_sum_fp64(f.s, f.t, s, t);
    out[4 * count + i] = c.s;
    out[5 * count + i] = c.t;
    out[6 * count + i] = s;
    out[7 * count + i] = t;
}

// The Strassen passes' DD addition with every error term on the integer pipe
// and dd_add (FP64 error terms) on the same operands
// (mpgemm_selftest_dd_add): in = [xh, xl, yh, yl] planes, out = [zh, zl] of
// dd_add_int, [zh, zl] of dd_add, and 1.0 where dd_add_int set `rare` (the
// passes recompute those with dd_add), else 0.0.
__global__ void k_selftest_dd_add(int64_t count, const double* in, double* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double* v = in + i;
    double zh, zl, fh, fl;
    bool rare = false;
    dd_add_int(v[0], v[count], v[2 * count], v[3 * count], zh, zl, rare);
    dd_add(v[0], v[count], v[2 * count], v[3 * count], fh, fl);
    out[i] = zh;
    out[count + i] = zl;
    out[2 * count + i] = fh;
    out[3 * count + i] = fl;
    out[4 * count + i] = rare ? 1.0 : 0.0;
}

}  // namespace mpg

extern "C" int mpgemm_selftest_dd_mac(int64_t count, const double* in, double* out, void* stream) {
    if (count < 0 || (count && (!in || !out))) return MPGEMM_EINVAL;
    if (count == 0) return MPGEMM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    mpg::PartitionScope pscope(st);
    mpg::k_selftest_dd_mac<<<mpg::ceil_div(count, 256), 256, 0, st>>>(count, in, out);
    return mpg::check_launch();
}

extern "C" int mpgemm_selftest_dd_add(int64_t count, const double* in, double* out, void* stream) {
    if (count < 0 || (count && (!in || !out))) return MPGEMM_EINVAL;
    if (count == 0) return MPGEMM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    mpg::PartitionScope pscope(st);
    mpg::k_selftest_dd_add<<<mpg::ceil_div(count, 256), 256, 0, st>>>(count, in, out);
    return mpg::check_launch();
}

extern "C" int mpgemm_selftest_two_prod(int64_t count, const double* a, const double* b, double* out,
                                        void* stream) {
    if (count < 0 || (count && (!a || !b || !out))) return MPGEMM_EINVAL;
    if (count == 0) return MPGEMM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    mpg::PartitionScope pscope(s);
    mpg::k_selftest_two_prod<<<mpg::ceil_div(count, 256), 256, 0, s>>>(count, a, b, out);
    return mpg::check_launch();
}

extern "C" int mpgemm_selftest_two_sum(int64_t count, const double* a, const double* b, double* out,
                                       void* stream) {
    if (count < 0 || (count && (!a || !b || !out))) return MPGEMM_EINVAL;
    if (count == 0) return MPGEMM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    mpg::PartitionScope pscope(s);
    mpg::k_selftest_two_sum<<<mpg::ceil_div(count, 256), 256, 0, s>>>(count, a, b, out);
    return mpg::check_launch();
}
