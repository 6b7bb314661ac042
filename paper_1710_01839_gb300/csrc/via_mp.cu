// DD and QD GEMMs on the integer pipe: the operands are rounded to p-bit
// multi-limb numbers, multiplied by the multi-limb GEMM (simple, block or
// Strassen, Eqs 1-3) and the product is rounded back to T doubles.
//
// Why: on GB300 the FP64 pipe delivers 2 operations per clock per SM
// (629 G op/s), while the integer pipes issue 128 thread-instructions per
// clock per SM.  A DD multiply-accumulate costs 5.1 FP64 operations (its
// product and error terms already on the integer pipe) and a QD one 51.25;
// a 128-bit multi-limb one about 232 integer instructions and a 256-bit one
// about 377, so the multi-limb path runs DD about 1.15x and QD about 6.5x
// faster, with every operation rounded to p >= 128 / 256 bits (far inside
// the DD and QD error bounds).
//
// Conversions (the definitions the oracle restates):
//   to p bits:   c = +0; for t = 0..T-1: c = RN_p(c + x_t), x_t taken exactly
//                (a double fits in p >= 64 bits);
//   from p bits: r = c; for t = 0..T-1: x_t = RN_53(r); r = r - x_t (exact),
//                i.e. the greedy expansion of the multi-limb value.
// Non-finite inputs set the invalid-input status bit; results outside the
// normal double range set the exponent-range bit.
#include "common.cuh"
#include "kernels.h"
#include "mp_arith.cuh"
#include "mp_convert.cuh"
#include "strassen.h"
#include "tune.h"

namespace mpg {

template <int W, int T>
__global__ void k_terms_to_mp(int64_t count, const double* __restrict__ X, uint32_t* __restrict__ Y,
                              unsigned* status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    unsigned st = 0u;
    MPV<W> c;
    terms_to_mp<W, T>(X + i, count, c, st);
    Y[i] = (uint32_t)c.e;
    Y[count + i] = c.f;
#pragma unroll
    for (int q = 0; q < W; q++) Y[(2 + q) * count + i] = c.m[q];
    if (st) atomicOr(status, st);
}

template <int W, int T>
__global__ void k_mp_to_terms(int64_t count, const uint32_t* __restrict__ Y, double* __restrict__ X,
                              unsigned* status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    unsigned st = 0u;
    MPV<W> r;
    r.e = (int)Y[i];
    r.f = Y[count + i];
#pragma unroll
    for (int q = 0; q < W; q++) r.m[q] = Y[(2 + q) * count + i];
    mp_to_terms<W, T>(r, X + i, count, st);
    if (st) atomicOr(status, st);
}

template <int W>
static int convert_w(int dir, int T, int64_t count, const double* X, uint32_t* Y, double* Xo, cudaStream_t s) {
    unsigned* status = device_status_ptr();
    if (!status) return MPGEMM_ECUDA;
    const unsigned grid = ceil_div(count, 128);
    if (dir == 0) {
        if (T == 2) k_terms_to_mp<W, 2><<<grid, 128, 0, s>>>(count, X, Y, status);
        else k_terms_to_mp<W, 4><<<grid, 128, 0, s>>>(count, X, Y, status);
    } else {
        if (T == 2) k_mp_to_terms<W, 2><<<grid, 128, 0, s>>>(count, Y, Xo, status);
        else k_mp_to_terms<W, 4><<<grid, 128, 0, s>>>(count, Y, Xo, status);
    }
    return check_launch();
}

// dir 0: T-term planes X (T x count doubles) -> multi-limb planes Y
// ((2 + w) x count words); dir 1: Y -> Xo.
static int convert(int dir, int T, int w, int64_t count, const double* X, uint32_t* Y, double* Xo, cudaStream_t s) {
    if (count == 0) return MPGEMM_OK;
    switch (w) {
        case 2: return convert_w<2>(dir, T, count, X, Y, Xo, s);
        case 4: return convert_w<4>(dir, T, count, X, Y, Xo, s);
        case 8: return convert_w<8>(dir, T, count, X, Y, Xo, s);
        case 16: return convert_w<16>(dir, T, count, X, Y, Xo, s);
        default: return MPGEMM_EUNSUPPORTED;
    }
}

static bool via_mp_width(int prec_bits, int* w) {
    if (prec_bits <= 0 || prec_bits % 32) return false;
    *w = prec_bits / 32;
    return *w == 2 || *w == 4 || *w == 8 || *w == 16;
}

static size_t mp_words(int w, int64_t r, int64_t c) { return (size_t)(2 + w) * (size_t)(r * c); }

size_t via_mp_workspace_bytes(int w, int64_t m, int64_t l, int64_t n, int algo, int depth) {
    size_t b = sizeof(uint32_t) * (mp_words(w, m, l) + mp_words(w, l, n) + mp_words(w, m, n));
    if (algo == MPGEMM_STRASSEN && depth > 0) b += strassen_workspace_bytes(sizeof(uint32_t) * (size_t)(2 + w), m, l, n, depth);
    return b;
}

static int via_mp_entry(int T, int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C,
                        int prec_bits, int algo, int n_min, int depth, void* stream) {
    int w = 0;
    if (!via_mp_width(prec_bits, &w)) return MPGEMM_EUNSUPPORTED;
    int rc = check_common(m, l, n, sizeof(double) * T, A, B, C, algo, n_min, depth);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    PartitionScope pscope(s);
    if (m == 0 || n == 0) return MPGEMM_OK;
    if (l == 0) {
        MPG_CUDA(cudaMemsetAsync(C, 0, sizeof(double) * (size_t)T * (size_t)(m * n), s));
        return MPGEMM_OK;
    }
    if (algo == MPGEMM_AUTO) {
        Choice ch;
        rc = auto_choice(MPGEMM_KIND_MP, prec_bits, m, l, n, stream_sms(s), &ch);
        if (rc) return rc;
        algo = ch.algo;
        n_min = ch.n_min;
        depth = ch.depth;
    }
    if (n_min <= 0) n_min = default_n_min(MPGEMM_KIND_MP);
    const bool strassen = algo == MPGEMM_STRASSEN && depth > 0;
    const size_t bytes = via_mp_workspace_bytes(w, m, l, n, strassen ? MPGEMM_STRASSEN : algo, depth);
    void* ws = nullptr;
    bool owned = false;
    rc = workspace_get(bytes, s, &ws, &owned);
    if (rc) return rc;
    uint32_t* Am = static_cast<uint32_t*>(ws);
    uint32_t* Bm = Am + mp_words(w, m, l);
    uint32_t* Cm = Bm + mp_words(w, l, n);
    uint32_t* rest = Cm + mp_words(w, m, n);
    rc = convert(0, T, w, m * l, A, Am, nullptr, s);
    if (!rc) rc = convert(0, T, w, l * n, B, Bm, nullptr, s);
    if (!rc) {
        CloseOperandsScope close;   // images of DD / QD numbers: operands of similar magnitude
        const size_t eb = sizeof(uint32_t) * (size_t)(2 + w);
        View<const uint32_t> a = bounded(planes_view<const uint32_t>(Am, m, l), Am, eb * m * l);
        View<const uint32_t> b = bounded(planes_view<const uint32_t>(Bm, l, n), Bm, eb * l * n);
        View<uint32_t> c = bounded(planes_view(Cm, m, n), Cm, eb * m * n);
        if (strassen) {
            const size_t sb = strassen_workspace_bytes(sizeof(uint32_t) * (size_t)(2 + w), m, l, n, depth);
            rc = strassen_mp_ws(w, m, l, n, a, b, c, n_min, depth, rest, sb, s);
        } else {
            rc = mp_gemm(w, algo == MPGEMM_SIMPLE ? MPGEMM_SIMPLE : MPGEMM_BLOCK, m, l, n, 1, a, b, c, n_min, s);
        }
    }
    if (!rc) rc = convert(1, T, w, m * n, nullptr, Cm, C, s);
    int rc2 = workspace_release(ws, owned, s);
    return rc ? rc : rc2;
}

}  // namespace mpg

using namespace mpg;

extern "C" {

int mpgemm_dd_via_mp(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int prec_bits,
                     int algo, int n_min, int strassen_depth, void* stream) {
    return via_mp_entry(2, m, l, n, A, B, C, prec_bits, algo, n_min, strassen_depth, stream);
}

int mpgemm_qd_via_mp(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int prec_bits,
                     int algo, int n_min, int strassen_depth, void* stream) {
    return via_mp_entry(4, m, l, n, A, B, C, prec_bits, algo, n_min, strassen_depth, stream);
}

size_t mpgemm_via_mp_workspace_size(int prec_bits, int64_t m, int64_t l, int64_t n, int algo, int strassen_depth) {
    int w = 0;
    if (!via_mp_width(prec_bits, &w) || m < 0 || l < 0 || n < 0) return 0;
    return via_mp_workspace_bytes(w, m, l, n, algo, strassen_depth);
}

int mpgemm_terms_to_mp(int terms, int64_t count, const double* X, int prec_bits, uint32_t* Y, void* stream) {
    int w = 0;
    if (terms != 2 && terms != 4) return MPGEMM_EINVAL;
    if (!via_mp_width(prec_bits, &w)) return MPGEMM_EUNSUPPORTED;
    if (count < 0 || (count && (!X || !Y))) return MPGEMM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    PartitionScope pscope(s);
    return convert(0, terms, w, count, X, Y, nullptr, s);
}

int mpgemm_mp_to_terms(int terms, int64_t count, int prec_bits, const uint32_t* Y, double* X, void* stream) {
    int w = 0;
    if (terms != 2 && terms != 4) return MPGEMM_EINVAL;
    if (!via_mp_width(prec_bits, &w)) return MPGEMM_EUNSUPPORTED;
    if (count < 0 || (count && (!X || !Y))) return MPGEMM_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    PartitionScope pscope(s);
    return convert(1, terms, w, count, nullptr, const_cast<uint32_t*>(Y), X, s);
}

}  // extern "C"
