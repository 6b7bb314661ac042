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
#include "kernels.h"
#include "profile.h"

namespace mpg {

struct DDFmt {
    static constexpr int P = 2;
    static constexpr int R = DD_RENORM;
    using Acc = DDAcc;
    __device__ static void zero(Acc& c) { dd_zero(c); }
    __device__ static void mac(Acc& c, const double* a, const double* b) { dd_mac(c, a[0], a[1], b[0], b[1]); }
    __device__ static void renorm(Acc& c) { dd_renorm(c); }
    __device__ static void finish(Acc& c, double* out) {
        double h, l;
        two_sum(c.s, c.t, h, l);
        out[0] = h;
        out[1] = l;
    }
};

struct QDFmt {
    static constexpr int P = 4;
    static constexpr int R = QD_RENORM;
    using Acc = QDAcc;
    __device__ static void zero(Acc& c) { qd_zero(c); }
    __device__ static void mac(Acc& c, const double* a, const double* b) { qd_mac(c, a, b); }
    __device__ static void renorm(Acc& c) { qd_renorm(c); }
    __device__ static void finish(Acc& c, double* out) {
        qd_finish(c);
        out[0] = c.s0;
        out[1] = c.s1;
        out[2] = c.s2;
        out[3] = c.s3;
    }
};

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
            a[q] = __ldg(pa + q * A.ps + k);
            b[q] = __ldg(pb + q * B.ps + k * B.ld);
        }
        Fmt::mac(acc, a, b);
        if ((k + 1) % Fmt::R == 0) Fmt::renorm(acc);
    }
    double out[P];
    Fmt::finish(acc, out);
#pragma unroll
    for (int q = 0; q < P; q++) *C.at(z, q, i, j) = out[q];
}

// ---------------------------------------------------------------- Eq 2

// One CTA computes a BM x BM block of C; each thread an RM x RM register
// tile (rows ty + r*TPD, columns tx + c*TPD).  K advances in panels of KT
// staged through shared memory as [k][row][plane].  CTA order follows the
// super-tile raster with group G (n_min / BM when n_min > BM).
template <class Fmt, int BM, int RM, int KT>
__global__ void __launch_bounds__((BM / RM) * (BM / RM)) k_block(int64_t m, int64_t l, int64_t n,
                                                                 View<const double> A, View<const double> B,
                                                                 View<double> C, unsigned G) {
    constexpr int P = Fmt::P;
    constexpr int TPD = BM / RM;
    constexpr int NT = TPD * TPD;
    constexpr int LD = (BM * KT) / NT;   // elements per thread per panel and operand
    static_assert((BM * KT) % NT == 0, "panel must split evenly over the threads");
    static_assert(KT % Fmt::R == 0, "renormalisation period must divide the panel depth");
    __shared__ __align__(16) double As[KT][BM][P];
    __shared__ __align__(16) double Bs[KT][BM][P];

    const unsigned tiles_m = ceil_div(m, BM), tiles_n = ceil_div(n, BM);
    unsigned tm, tn;
    raster(blockIdx.x, tiles_m, tiles_n, G, tm, tn);
    const int64_t z = blockIdx.y;
    const int64_t i0 = (int64_t)tm * BM, j0 = (int64_t)tn * BM;
    const int tid = threadIdx.x;
    const int ty = tid / TPD, tx = tid % TPD;

    typename Fmt::Acc acc[RM][RM];
#pragma unroll
    for (int r = 0; r < RM; r++)
#pragma unroll
        for (int c = 0; c < RM; c++) Fmt::zero(acc[r][c]);

    double ra[LD][P], rb[LD][P];
    auto gload = [&](int64_t k0) {
#pragma unroll
        for (int v = 0; v < LD; v++) {
            int idx = tid + v * NT;
            int r = idx / KT, c = idx % KT;          // A panel: BM rows x KT
            int64_t i = i0 + r, k = k0 + c;
            bool ok = i < m && k < l;
#pragma unroll
            for (int q = 0; q < P; q++) ra[v][q] = ok ? __ldg(A.at(z, q, i, k)) : 0.0;
            int rr = idx / BM, cc = idx % BM;        // B panel: KT rows x BM
            int64_t kb = k0 + rr, j = j0 + cc;
            bool okb = kb < l && j < n;
#pragma unroll
            for (int q = 0; q < P; q++) rb[v][q] = okb ? __ldg(B.at(z, q, kb, j)) : 0.0;
        }
    };
    auto sstore = [&]() {
#pragma unroll
        for (int v = 0; v < LD; v++) {
            int idx = tid + v * NT;
            int r = idx / KT, c = idx % KT;
            int rr = idx / BM, cc = idx % BM;
#pragma unroll
            for (int q = 0; q < P; q++) {
                As[c][r][q] = ra[v][q];
                Bs[rr][cc][q] = rb[v][q];
            }
        }
    };

    gload(0);
    sstore();
    __syncthreads();
    for (int64_t k0 = 0; k0 < l; k0 += KT) {
        const bool more = k0 + KT < l;
        if (more) gload(k0 + KT);
#pragma unroll
        for (int kk = 0; kk < KT; kk++) {
            double a[RM][P], b[RM][P];
#pragma unroll
            for (int r = 0; r < RM; r++)
#pragma unroll
                for (int q = 0; q < P; q++) a[r][q] = As[kk][ty + r * TPD][q];
#pragma unroll
            for (int c = 0; c < RM; c++)
#pragma unroll
                for (int q = 0; q < P; q++) b[c][q] = Bs[kk][tx + c * TPD][q];
#pragma unroll
            for (int r = 0; r < RM; r++)
#pragma unroll
                for (int c = 0; c < RM; c++) Fmt::mac(acc[r][c], a[r], b[c]);
            if ((kk + 1) % Fmt::R == 0) {
#pragma unroll
                for (int r = 0; r < RM; r++)
#pragma unroll
                    for (int c = 0; c < RM; c++) Fmt::renorm(acc[r][c]);
            }
        }
        __syncthreads();
        if (more) {
            sstore();
            __syncthreads();
        }
    }

#pragma unroll
    for (int r = 0; r < RM; r++)
#pragma unroll
        for (int c = 0; c < RM; c++) {
            int64_t i = i0 + ty + r * TPD, j = j0 + tx + c * TPD;
            double out[P];
            Fmt::finish(acc[r][c], out);
            if (i < m && j < n) {
#pragma unroll
                for (int q = 0; q < P; q++) *C.at(z, q, i, j) = out[q];
            }
        }
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

}  // namespace mpg
