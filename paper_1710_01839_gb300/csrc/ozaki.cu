// Split-precision DD GEMM (Ozaki-style) on the INT8 tensor path.
//
//  1. e_i = max_k expo(hi(a_ik)), f_j = max_k expo(hi(b_kj)) (frexp exponent).
//  2. Digits: T = trunc((a_ik) 2^(7S - e_i)) toward zero, an exact integer of
//     at most 7S bits, split into S signed base-128 digits d_1..d_S (int8 in
//     [-127, 127], most significant first).  Computed from the two words
//     with integer arithmetic: no FP64 loop per digit.
//  3. Level sums L_g = sum_{s+t=g} D_s^A (D_t^B)^T for g = 2..S+1 (the
//     triangle s + t <= S + 1), int8 x int8 -> int32 on the tensor cores
//     (mma.sync m16n8k32 s8: sm_103a has no tcgen05 integer MMA), exact.
//  4. c_ij = RN_DD(2^(e_i + f_j) sum_g L_g 2^(-7g)): the level sums are added
//     exactly in a 192-bit integer and rounded once to (hi, lo) =
//     (RN(x), RN(x - RN(x))), so every step is exact up to that final
//     rounding and the result is bit-identical to the definition.
#include <climits>
#include <cstdint>

#include "common.cuh"
#include "ozaki.h"
#include "ozaki_digits.cuh"
#include "profile.h"
#include "strassen.h"
#include "tc_levels.h"

namespace mpg {

// ---------------------------------------------------------------- step 1

__device__ __forceinline__ int expo_of(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    // +-0, tested on the 32-bit halves (a test on the 64-bit pattern can
    // become an FP64 compare, which takes the slow FP64 pipe)
    if ((((unsigned)__double2hiint(x) << 1) | (unsigned)__double2loint(x)) == 0u) return INT_MIN;
    int E = (int)((b >> 52) & 0x7ff);
    if (E == 0) {   // subnormal: 0.m * 2^-1022, leading one of m decides
        unsigned long long mant = b & ((1ull << 52) - 1);
        return -1022 - (__clzll(mant) - 12);
    }
    return E - 1022;
}

// One warp per row of the hi plane.
__global__ void k_row_expo(int64_t m, int64_t l, const double* hi, int* e) {
    int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    int lane = threadIdx.x & 31;
    if (row >= m) return;
    int mx = INT_MIN;
    for (int64_t k = lane; k < l; k += 32) mx = max(mx, expo_of(hi[row * l + k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) e[row] = mx == INT_MIN ? 0 : mx;
}

// Column maxima in parallel over rows: a block covers 32 columns x
// COLX_ROWS rows (a warp reads 32 consecutive doubles of one row) and
// atomically raises f[j], pre-filled with COLX_EMPTY, which lies below every
// finite frexp exponent (>= -1073) and above the INT_MIN of a zero element.
constexpr int COLX_ROWS = 256;
constexpr int COLX_EMPTY = (int)0x80808080;   // the byte fill 0x80
__global__ void k_col_expo(int64_t l, int64_t n, const double* hi, int* f) {
    const int64_t j = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t k0 = (int64_t)blockIdx.y * COLX_ROWS;
    if (j >= n) return;
    const int64_t k1 = k0 + COLX_ROWS < l ? k0 + COLX_ROWS : l;
    int mx = INT_MIN;
#pragma unroll 4
    for (int64_t k = k0 + threadIdx.y; k < k1; k += blockDim.y) mx = max(mx, expo_of(hi[k * n + j]));
    __shared__ int red[8][32];
    red[threadIdx.y][threadIdx.x] = mx;
    __syncthreads();
    if (threadIdx.y == 0) {
        for (int y = 1; y < (int)blockDim.y; y++) mx = max(mx, red[y][threadIdx.x]);
        if (mx != INT_MIN) atomicMax(f + j, mx);
    }
}
// An all-zero column keeps the fill value: its exponent is 0.
__global__ void k_expo_fix(int64_t n, int* f) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n && f[j] == COLX_EMPTY) f[j] = 0;
}

// ---------------------------------------------------------------- step 2

// |x| of an integer-valued double as a 128-bit integer (hi:lo).
__device__ __forceinline__ void dbl_int_to_u128(double x, unsigned long long& hi, unsigned long long& lo) {
    double a = fabs(x);
    hi = lo = 0ull;
    if (a == 0.0) return;
    unsigned long long b = (unsigned long long)__double_as_longlong(a);
    int E = (int)(b >> 52);
    unsigned long long M = (b & ((1ull << 52) - 1)) | (1ull << 52);
    int sh = E - 1075;   // a = M 2^sh, and a integer => sh >= 0 or low bits of M are zero
    if (sh < 0) {
        lo = M >> (-sh);
        return;
    }
    if (sh == 0) {
        lo = M;
    } else if (sh < 64) {
        lo = M << sh;
        hi = M >> (64 - sh);
    } else {
        hi = M << (sh - 64);
    }
}

__device__ __forceinline__ void add_s128(unsigned long long& hi, unsigned long long& lo, bool neg_a,
                                         unsigned long long bh, unsigned long long bl, bool neg_b, bool& neg_out) {
    // (neg_a ? -A : A) + (neg_b ? -B : B) in sign-magnitude, |result| < 2^127
    if (neg_a == neg_b) {
        unsigned long long l2 = lo + bl;
        hi = hi + bh + (l2 < lo ? 1ull : 0ull);
        lo = l2;
        neg_out = neg_a;
        return;
    }
    bool a_ge = hi > bh || (hi == bh && lo >= bl);
    if (a_ge) {
        unsigned long long l2 = lo - bl;
        hi = hi - bh - (lo < bl ? 1ull : 0ull);
        lo = l2;
        neg_out = neg_a;
    } else {
        unsigned long long l2 = bl - lo;
        hi = bh - hi - (bl < lo ? 1ull : 0ull);
        lo = l2;
        neg_out = neg_b;
    }
}

// Digits of trunc((hi + lo) 2^(7S - e)) (exact; |value| < 2^e so |T| < 2^(7S)).
__device__ __forceinline__ void dd_digits(double hi, double lo, int e, int S, signed char* d, int64_t stride) {
    const int sc = 7 * S - e;
    double H = ldexp(hi, sc), L = ldexp(lo, sc);   // exact power-of-two scalings
    double tH = trunc(H);
    double corr = 0.0;
    if (tH == H) {
        // H an integer: L (|L| <= ulp(H)/2) decides whether H + L crosses it
        if (H > 0.0 && L < 0.0) corr = floor(L);
        else if (H < 0.0 && L > 0.0) corr = ceil(L);
        else corr = trunc(L);
    }
    unsigned long long th, tl, ch, cl;
    dbl_int_to_u128(tH, th, tl);
    dbl_int_to_u128(corr, ch, cl);
    bool neg;
    add_s128(th, tl, tH < 0.0, ch, cl, corr < 0.0, neg);
    for (int s = 0; s < S; s++) {
        int sh = 7 * (S - 1 - s);
        unsigned long long v = sh >= 64 ? (th >> (sh - 64)) : (sh == 0 ? tl : ((tl >> sh) | (th << (64 - sh))));
        int dig = (int)(v & 127ull);
        d[(int64_t)s * stride] = (signed char)(neg ? -dig : dig);
    }
}

// Two e4m3 codes of small integers in one instruction (exact for |v| <= 16):
// the low byte holds a, the high byte b.
__device__ __forceinline__ unsigned e4m3x2_of(int a, int b) {
    unsigned short r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"((float)b), "f"((float)a));
    return (unsigned)r;
}

template <int K>
__device__ __forceinline__ int b32_digit(const B32& u, int S) {
    const int d = b32_field<K>(u) - (K < S - 1 ? 16 : 0);
    return u.neg ? -d : d;
}

// Digit k of four consecutive elements as four e4m3 codes (element 0 in the low byte).
template <int K>
__device__ __forceinline__ unsigned b32_word(const B32 (&u)[4], int S) {
    return e4m3x2_of(b32_digit<K>(u[0], S), b32_digit<K>(u[1], S)) |
           (e4m3x2_of(b32_digit<K>(u[2], S), b32_digit<K>(u[3], S)) << 16);
}

// Calls f(K, word) for K = 0 .. S-1 (S <= 24), K compile-time.
template <int K, typename F>
__device__ __forceinline__ void b32_words(const B32 (&u)[4], int S, F&& f) {
    if constexpr (K < 24) {
        if (K < S) {
            f(K, b32_word<K>(u, S));
            b32_words<K + 1>(u, S, f);
        }
    }
}

// A (m x l, row scale e): digits into S planes of m x lp.  One thread per
// four consecutive K positions: 4-byte stores, a warp writes 128 contiguous
// bytes of every plane.  Positions l <= k < lp are written as zero digits.
__global__ void k_slice_rows_f8(int64_t m, int64_t l, int64_t lp, const double* A, const int* e, int S,
                                unsigned long long Ch, unsigned long long Cl, int vec, unsigned char* D) {
    const int64_t k0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    const int64_t i = blockIdx.y;
    if (k0 >= lp || i >= m) return;
    const int sc = 5 * S - e[i] - 1;
    const double* hiA = A + i * l;
    const double* loA = A + m * l + i * l;
    double h[4], o[4];
    if (vec && k0 + 4 <= l) {   // vec: A 16-byte aligned and l even
        const double2 h01 = *(const double2*)(hiA + k0), h23 = *(const double2*)(hiA + k0 + 2);
        const double2 o01 = *(const double2*)(loA + k0), o23 = *(const double2*)(loA + k0 + 2);
        h[0] = h01.x; h[1] = h01.y; h[2] = h23.x; h[3] = h23.y;
        o[0] = o01.x; o[1] = o01.y; o[2] = o23.x; o[3] = o23.y;
    } else {
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const bool in = k0 + t < l;
            h[t] = in ? hiA[k0 + t] : 0.0;
            o[t] = in ? loA[k0 + t] : 0.0;
        }
    }
    B32 u[4];
#pragma unroll
    for (int t = 0; t < 4; t++) u[t] = b32_prepare(h[t], o[t], sc, Ch, Cl);
    const int64_t plane = m * lp;
    unsigned* out = (unsigned*)(D + i * lp + k0);
    b32_words<0>(u, S, [&](int K, unsigned w) { out[(int64_t)(S - 1 - K) * (plane >> 2)] = w; });
}

// B (l x n, column scale f): digits transposed into S planes of n x lp.  A
// block of 128 threads covers 32 columns x 64 rows of B: lane t takes column
// j0 + t (a warp reads 256 contiguous bytes of a row), warp w rows k0 + 4q
// .. + 3 for q = w, w + 4, w + 8, w + 12; the digit words go through shared
// memory (rows of 16 words padded to 17: conflict-free) and leave as 64-byte
// row segments of each plane.
constexpr int SLC_COLS = 32, SLC_ROWS = 64, SLC_PITCH = SLC_ROWS / 4 + 1;
__global__ void __launch_bounds__(128) k_slice_cols_f8(int64_t l, int64_t n, int64_t lp, const double* B,
                                                       const int* f, int S, unsigned long long Ch,
                                                       unsigned long long Cl, unsigned char* D) {
    extern __shared__ unsigned tile[];   // [S][SLC_COLS][SLC_PITCH]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k0 = (int64_t)blockIdx.x * SLC_ROWS, j0 = (int64_t)blockIdx.y * SLC_COLS;
    const int64_t j = j0 + lane;
    const bool jin = j < n;
    const int sc = 5 * S - (jin ? f[j] : 0) - 1;
    const double* loB = B + l * n;
#pragma unroll 1
    for (int q = warp; q < SLC_ROWS / 4; q += 4) {
        B32 u[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const int64_t k = k0 + 4 * q + t;
            const bool in = jin && k < l;
            u[t] = b32_prepare(in ? B[k * n + j] : 0.0, in ? loB[k * n + j] : 0.0, sc, Ch, Cl);
        }
        b32_words<0>(u, S, [&](int K, unsigned w) { tile[((S - 1 - K) * SLC_COLS + lane) * SLC_PITCH + q] = w; });
    }
    __syncthreads();
    const int64_t plane = n * lp;
    for (int s = 0; s < S; s++) {
#pragma unroll
        for (int r = 0; r < (SLC_COLS * SLC_ROWS / 4) / 128; r++) {
            const int idx = threadIdx.x + 128 * r, row = idx >> 4, w = idx & 15;
            const int64_t jj = j0 + row, kk = k0 + 4 * w;
            if (jj < n && kk < lp)
                *(unsigned*)(D + (int64_t)s * plane + jj * lp + kk) = tile[(s * SLC_COLS + row) * SLC_PITCH + w];
        }
    }
}


// ---- FP8 digits of T-term expansions (QD, T = 4): the same scheme with the
// exact truncation on NW = 4 64-bit words and up to QD_SMAX digits.
constexpr int QD_SMAX = 48;   // 5 S + 1 bits of the biased value stay below 2^256

struct Bias4 {
    unsigned long long w[4];
};

template <int K>
__device__ __forceinline__ int b32_digit_q(const WideB32<4>& u, int S) {
    const int d = b32_field_wide<K, 4>(u) - (K < S - 1 ? 16 : 0);
    return u.neg ? -d : d;
}

template <int K>
__device__ __forceinline__ unsigned b32_word_q(const WideB32<4> (&u)[4], int S) {
    return e4m3x2_of(b32_digit_q<K>(u[0], S), b32_digit_q<K>(u[1], S)) |
           (e4m3x2_of(b32_digit_q<K>(u[2], S), b32_digit_q<K>(u[3], S)) << 16);
}

template <int K, typename F>
__device__ __forceinline__ void b32_words_q(const WideB32<4> (&u)[4], int S, F&& f) {
    if constexpr (K < QD_SMAX) {
        if (K < S) {
            f(K, b32_word_q<K>(u, S));
            b32_words_q<K + 1>(u, S, f);
        }
    }
}

template <int T>
__device__ __forceinline__ void prepare_q(const double (&x)[T], int sc, const Bias4& C, WideB32<4>& u) {
    expansion_trunc_scaled<T, 4>(x, sc, u);
    const unsigned long long c[4] = {C.w[0], C.w[1], C.w[2], C.w[3]};
    b32_prepare_wide<4>(u, c);
}

// A (T planes of m x l, row scale e): digits into S planes of m x lp, four
// consecutive K positions per thread (one 32-bit store per plane).
template <int T>
__global__ void k_slice_rows_f8_terms(int64_t m, int64_t l, int64_t lp, const double* X, const int* e, int S,
                                      Bias4 C, unsigned char* D) {
    const int64_t k0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    const int64_t i = blockIdx.y;
    if (k0 >= lp || i >= m) return;
    const int sc = 5 * S - e[i] - 1;
    const int64_t plane_in = m * l;
    WideB32<4> u[4];
#pragma unroll
    for (int t = 0; t < 4; t++) {
        double x[T];
#pragma unroll
        for (int q = 0; q < T; q++) x[q] = k0 + t < l ? X[q * plane_in + i * l + k0 + t] : 0.0;
        prepare_q<T>(x, sc, C, u[t]);
    }
    const int64_t plane = m * lp;
    unsigned* out = (unsigned*)(D + i * lp + k0);
    b32_words_q<0>(u, S, [&](int K, unsigned w) { out[(int64_t)(S - 1 - K) * (plane >> 2)] = w; });
}

// B (T planes of l x n, column scale f): digits transposed into S planes of
// n x lp through shared memory, as k_slice_cols_f8 does for DD.
template <int T>
__global__ void __launch_bounds__(128) k_slice_cols_f8_terms(int64_t l, int64_t n, int64_t lp, const double* X,
                                                             const int* f, int S, Bias4 C, unsigned char* D) {
    extern __shared__ unsigned tile[];   // [S][SLC_COLS][SLC_PITCH]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k0 = (int64_t)blockIdx.x * SLC_ROWS, j0 = (int64_t)blockIdx.y * SLC_COLS;
    const int64_t j = j0 + lane;
    const bool jin = j < n;
    const int sc = 5 * S - (jin ? f[j] : 0) - 1;
    const int64_t plane_in = l * n;
#pragma unroll 1
    for (int q4 = warp; q4 < SLC_ROWS / 4; q4 += 4) {
        WideB32<4> u[4];
#pragma unroll
        for (int t = 0; t < 4; t++) {
            const int64_t k = k0 + 4 * q4 + t;
            const bool in = jin && k < l;
            double x[T];
#pragma unroll
            for (int q = 0; q < T; q++) x[q] = in ? X[q * plane_in + k * n + j] : 0.0;
            prepare_q<T>(x, sc, C, u[t]);
        }
        b32_words_q<0>(u, S, [&](int K, unsigned w) { tile[((S - 1 - K) * SLC_COLS + lane) * SLC_PITCH + q4] = w; });
    }
    __syncthreads();
    const int64_t plane = n * lp;
    for (int s = 0; s < S; s++) {
#pragma unroll
        for (int r = 0; r < (SLC_COLS * SLC_ROWS / 4) / 128; r++) {
            const int idx = threadIdx.x + 128 * r, row = idx >> 4, w = idx & 15;
            const int64_t jj = j0 + row, kk = k0 + 4 * w;
            if (jj < n && kk < lp)
                *(unsigned*)(D + (int64_t)s * plane + jj * lp + kk) = tile[(s * SLC_COLS + row) * SLC_PITCH + w];
        }
    }
}

// A (m x l, row scale e): digits into S planes of m x lp (K contiguous, zero padded).
__global__ void k_slice_rows(int64_t m, int64_t l, int64_t lp, const double* A, const int* e, int S, signed char* D) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = blockIdx.y;
    if (k >= lp || i >= m) return;
    signed char* out = D + i * lp + k;
    const int64_t plane = m * lp;
    if (k >= l) {
        for (int s = 0; s < S; s++) out[s * plane] = 0;
        return;
    }
    const int64_t idx = i * l + k;
    dd_digits(A[idx], A[m * l + idx], e[i], S, out, plane);
}

// B (l x n, column scale f): digits into S planes of n x lp (transposed: K contiguous).
__global__ void k_slice_cols(int64_t l, int64_t n, int64_t lp, const double* B, const int* f, int S, signed char* D) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t j = blockIdx.y;
    if (k >= lp || j >= n) return;
    signed char* out = D + j * lp + k;
    const int64_t plane = n * lp;
    if (k >= l) {
        for (int s = 0; s < S; s++) out[s * plane] = 0;
        return;
    }
    const int64_t idx = k * n + j;
    dd_digits(B[idx], B[l * n + idx], f[j], S, out, plane);
}

// ---------------------------------------------------------------- step 3

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}
__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void* smem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}
__device__ __forceinline__ void mma_s8(int (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr int OZ_BM = 128, OZ_BN = 128, OZ_BK = 64, OZ_STAGES = 4, OZ_THREADS = 256;
constexpr int OZ_STAGE_BYTES = (OZ_BM + OZ_BN) * OZ_BK;   // 16 KB
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE_BYTES;       // 64 KB

// 16-byte chunk c (0..3) of smem row r, XOR-swizzled so that ldmatrix's
// eight row reads of one 16-byte column hit eight different bank groups.
__device__ __forceinline__ int swz(int r, int c) { return r * OZ_BK + ((c ^ ((r >> 1) & 3)) << 4); }

// One CTA = one 128 x 128 tile of one level g; levels are issued heaviest
// first (level g concatenates g - 1 slice pairs along K).  8 warps as 2 x 4,
// warp tile 64 x 32 = 4 x 4 mma tiles; 4-stage cp.async pipeline; int8
// digits, s32 accumulators.  (FP8 digits run on the tcgen05 kernel of
// tc_levels.cu.)
__global__ void __launch_bounds__(OZ_THREADS) k_ozaki_levels(int64_t m, int64_t n, int64_t lp, int S,
                                                             const unsigned char* DA, const unsigned char* DB,
                                                             int* Lv, unsigned tiles_m, unsigned tiles_n) {
    extern __shared__ __align__(128) unsigned char smem[];
    const unsigned tiles = tiles_m * tiles_n;
    const unsigned gi = blockIdx.x / tiles, tile = blockIdx.x % tiles;
    const int g = S + 1 - (int)gi;
    const unsigned tm = tile / tiles_n, tn = tile % tiles_n;
    const int64_t row0 = (int64_t)tm * OZ_BM, col0 = (int64_t)tn * OZ_BN;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 2, wn = warp & 3;
    const int ksteps = (int)(lp / OZ_BK);
    const int total = (g - 1) * ksteps;
    const int64_t planeA = m * lp, planeB = n * lp;

    auto load = [&](int it, int stage) {
        int s = it / ksteps + 1;
        int64_t kb = (int64_t)(it % ksteps) * OZ_BK;
        const unsigned char* Ab = DA + (int64_t)(s - 1) * planeA + kb;
        const unsigned char* Bb = DB + (int64_t)(g - s - 1) * planeB + kb;
        unsigned char* sA = smem + stage * OZ_STAGE_BYTES;
        unsigned char* sB = sA + OZ_BM * OZ_BK;
#pragma unroll
        for (int v = 0; v < 2; v++) {
            int cid = tid + OZ_THREADS * v;
            int r = cid >> 2, c = cid & 3;
            int64_t ga = row0 + r, gb = col0 + r;
            bool va = ga < m, vb = gb < n;
            cp_async16(sA + swz(r, c), va ? (const void*)(Ab + ga * lp + c * 16) : (const void*)DA, va ? 16 : 0);
            cp_async16(sB + swz(r, c), vb ? (const void*)(Bb + gb * lp + c * 16) : (const void*)DB, vb ? 16 : 0);
        }
    };

    int acc[4][4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[a][b][c] = 0;

#pragma unroll
    for (int st = 0; st < OZ_STAGES - 1; st++) {
        if (st < total) load(st, st);
        cp_async_commit();
    }
    for (int it = 0; it < total; it++) {
        cp_async_wait<OZ_STAGES - 2>();
        __syncthreads();
        int nx = it + OZ_STAGES - 1;
        if (nx < total) load(nx, nx % OZ_STAGES);
        cp_async_commit();
        const unsigned char* sA = smem + (it % OZ_STAGES) * OZ_STAGE_BYTES;
        const unsigned char* sB = sA + OZ_BM * OZ_BK;
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {
            unsigned a[4][4], b[2][4];
#pragma unroll
            for (int mi = 0; mi < 4; mi++) {
                int r = wm * 64 + mi * 16 + (lane & 15);
                ldsm_x4(a[mi], sA + swz(r, ks * 2 + (lane >> 4)));
            }
#pragma unroll
            for (int nj = 0; nj < 2; nj++) {
                int q = lane >> 3;
                int r = wn * 32 + nj * 16 + (lane & 7) + 8 * (q >> 1);
                ldsm_x4(b[nj], sB + swz(r, ks * 2 + (q & 1)));
            }
#pragma unroll
            for (int mi = 0; mi < 4; mi++)
#pragma unroll
                for (int ni = 0; ni < 4; ni++)
                    mma_s8(acc[mi][ni], a[mi], b[ni >> 1][(ni & 1) * 2], b[ni >> 1][(ni & 1) * 2 + 1]);
        }
    }
    cp_async_wait<0>();

    int* out = Lv + (int64_t)(g - 2) * m * n;
    const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 4; mi++)
#pragma unroll
        for (int ni = 0; ni < 4; ni++) {
            int64_t c = col0 + wn * 32 + ni * 8 + 2 * tq;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                int64_t r = row0 + wm * 64 + mi * 16 + gq + 8 * h;
                if (r < m) {
                    if (c < n) out[r * n + c] = acc[mi][ni][2 * h];
                    if (c + 1 < n) out[r * n + c + 1] = acc[mi][ni][2 * h + 1];
                }
            }
        }
}

// ---------------------------------------------------------------- step 4

// V += x (a sign-extended int64) on NL 32-bit limbs, one carry chain.
template <int NL>
__device__ __forceinline__ void limbs_add_i64(uint32_t (&w)[NL], long long x);
template <>
__device__ __forceinline__ void limbs_add_i64<6>(uint32_t (&w)[6], long long x) {
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)((unsigned long long)x >> 32), ext = (uint32_t)(x >> 63);
    asm("add.cc.u32 %0, %0, %6;\n\taddc.cc.u32 %1, %1, %7;\n\taddc.cc.u32 %2, %2, %8;\n\t"
        "addc.cc.u32 %3, %3, %8;\n\taddc.cc.u32 %4, %4, %8;\n\taddc.u32 %5, %5, %8;"
        : "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3]), "+r"(w[4]), "+r"(w[5])
        : "r"(lo), "r"(hi), "r"(ext));
}
template <>
__device__ __forceinline__ void limbs_add_i64<10>(uint32_t (&w)[10], long long x) {
    const uint32_t lo = (uint32_t)x, hi = (uint32_t)((unsigned long long)x >> 32), ext = (uint32_t)(x >> 63);
    asm("add.cc.u32 %0, %0, %10;\n\taddc.cc.u32 %1, %1, %11;\n\taddc.cc.u32 %2, %2, %12;\n\t"
        "addc.cc.u32 %3, %3, %12;\n\taddc.cc.u32 %4, %4, %12;\n\taddc.cc.u32 %5, %5, %12;\n\t"
        "addc.cc.u32 %6, %6, %12;\n\taddc.cc.u32 %7, %7, %12;\n\taddc.cc.u32 %8, %8, %12;\n\t"
        "addc.u32 %9, %9, %12;"
        : "+r"(w[0]), "+r"(w[1]), "+r"(w[2]), "+r"(w[3]), "+r"(w[4]), "+r"(w[5]), "+r"(w[6]), "+r"(w[7]),
          "+r"(w[8]), "+r"(w[9])
        : "r"(lo), "r"(hi), "r"(ext));
}

// V = sum_{g=2}^{S+1} L_g 2^(BITS (S + 1 - g)) as NW 64-bit words (two's
// complement), computed on 2 NW 32-bit limbs.  Levels go in groups of G
// (G BITS <= 30): a group's sum sum_j L_{g0+j} 2^(BITS (G' - 1 - j)) is
// exact in an int64 (|L_g| < 2^31), then V <- V 2^(BITS G') + group with
// funnel shifts and one carry chain; a group's loads are issued together.
// Used for QD (10 limbs), where it cuts the wide steps by G; the DD kernel
// keeps one level per step (measured faster on 6 limbs).
template <int BITS, int NW, int G>
__device__ __forceinline__ void horner_levels(const int* __restrict__ lp, int64_t mn, int S,
                                              unsigned long long (&v)[NW]) {
    static_assert(G >= 1 && G * BITS <= 30, "group shift must stay within one limb");
    constexpr int NL = 2 * NW;
    uint32_t w[NL];
#pragma unroll
    for (int q = 0; q < NL; q++) w[q] = 0u;
    for (int g0 = 2; g0 <= S + 1; g0 += G) {
        const int cnt = (S + 2 - g0) < G ? (S + 2 - g0) : G;
        int x[G];
#pragma unroll
        for (int j = 0; j < G; j++) {   // unconditional loads (clamped plane), zeroed past the group
            const int gi = (g0 - 2 + j) < S - 1 ? (g0 - 2 + j) : S - 1;
            x[j] = lp[(int64_t)gi * mn];
        }
#pragma unroll
        for (int j = 0; j < G; j++) x[j] = j < cnt ? x[j] : 0;
        long long grp = 0;
#pragma unroll
        for (int j = 0; j < G; j++)
            if (j < cnt) grp = (long long)((unsigned long long)grp << BITS) + x[j];
        const int sh = BITS * cnt;   // <= 30
#pragma unroll
        for (int q = NL - 1; q > 0; q--) w[q] = __funnelshift_l(w[q - 1], w[q], sh);
        w[0] <<= sh;
        limbs_add_i64<NL>(w, grp);
    }
#pragma unroll
    for (int q = 0; q < NW; q++) v[q] = ((unsigned long long)w[2 * q + 1] << 32) | w[2 * q];
}

// v (192-bit two's complement, 3 limbs) += x * 2^sh, 0 <= sh < 128.
__device__ __forceinline__ void add_shifted(unsigned long long (&v)[3], long long x, int sh) {
    unsigned long long w0 = (unsigned long long)x, ext = x < 0 ? ~0ull : 0ull;
    unsigned long long t[3];
    if (sh == 0) {
        t[0] = w0; t[1] = ext; t[2] = ext;
    } else if (sh < 64) {
        t[0] = w0 << sh;
        t[1] = (w0 >> (64 - sh)) | (ext << sh);
        t[2] = ext;
    } else if (sh == 64) {
        t[0] = 0; t[1] = w0; t[2] = ext;
    } else {
        int r = sh - 64;
        t[0] = 0;
        t[1] = w0 << r;
        t[2] = (w0 >> (64 - r)) | (ext << r);
    }
    unsigned long long c = 0;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        unsigned long long s1 = v[i] + t[i];
        unsigned long long c1 = s1 < v[i] ? 1ull : 0ull;
        unsigned long long s2 = s1 + c;
        unsigned long long c2 = s2 < s1 ? 1ull : 0ull;
        v[i] = s2;
        c = c1 | c2;
    }
}

__device__ __forceinline__ int top_bit(const unsigned long long (&u)[3]) {
    if (u[2]) return 128 + 63 - __clzll(u[2]);
    if (u[1]) return 64 + 63 - __clzll(u[1]);
    if (u[0]) return 63 - __clzll(u[0]);
    return -1;
}
__device__ __forceinline__ unsigned long long bits_at(const unsigned long long (&u)[3], int lo, int cnt) {
    // bits [lo, lo + cnt) (cnt <= 64, lo >= 0)
    int q = lo >> 6, r = lo & 63;
    unsigned long long a = q < 3 ? u[q] : 0ull, b = q + 1 < 3 ? u[q + 1] : 0ull;
    unsigned long long v = r ? ((a >> r) | (b << (64 - r))) : a;
    return cnt >= 64 ? v : (v & ((1ull << cnt) - 1ull));
}
__device__ __forceinline__ bool any_below(const unsigned long long (&u)[3], int pos) {
    int q = pos >> 6, r = pos & 63;
    for (int i = 0; i < q && i < 3; i++)
        if (u[i]) return true;
    return q < 3 && r && (u[q] & ((1ull << r) - 1ull));
}

// Round |u| (u >= 0) to 53 bits, ties to even: returns mantissa M and the
// position t - 52 of its last bit (value ~= M 2^(t-52)); M == 0 for u == 0.
__device__ __forceinline__ unsigned long long rn53(const unsigned long long (&u)[3], int& pos) {
    int t = top_bit(u);
    if (t < 0) {
        pos = 0;
        return 0ull;
    }
    if (t <= 52) {
        pos = 0;
        return u[0];
    }
    unsigned long long M = bits_at(u, t - 52, 53);
    bool rb = bits_at(u, t - 53, 1) != 0ull;
    bool st = any_below(u, t - 53);
    if (rb && (st || (M & 1ull))) M += 1ull;
    pos = t - 52;
    return M;
}

__device__ __forceinline__ void neg192(unsigned long long (&v)[3]) {
    unsigned long long c = 1;
#pragma unroll
    for (int i = 0; i < 3; i++) {
        unsigned long long x = ~v[i] + c;
        c = (c && x == 0ull) ? 1ull : 0ull;
        v[i] = x;
    }
}

// bits = digit width (7 for int8, 5 for e4m3), head = headroom bits per side
// (0 for int8, 1 for e4m3): x = 2^(e_i + f_j + 2 head) sum_g L_g 2^(-bits g).
template <int BITS>
__global__ void k_recombine(int64_t m, int64_t n, int S, int head, const int* Lv, const int* e, const int* f,
                            double* C) {
    constexpr int bits = BITS;
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = blockIdx.y;
    if (j >= n) return;
    const int64_t mn = m * n, idx = i * n + j;
    // V = sum_g L_g 2^(bits (S + 1 - g)) by Horner's rule, V <- V 2^bits + L_g,
    // on six 32-bit limbs (two's complement; |L_g| < 2^31 gives |V| < 2^(32 + bits (S - 1)) <= 2^151)
    unsigned w0 = 0, w1 = 0, w2 = 0, w3 = 0, w4 = 0, w5 = 0;
    const int* lp = Lv + idx;
#pragma unroll 4
    for (int g = 2; g <= S + 1; g++) {
        const int x = lp[(int64_t)(g - 2) * mn];
        w5 = __funnelshift_l(w4, w5, bits);
        w4 = __funnelshift_l(w3, w4, bits);
        w3 = __funnelshift_l(w2, w3, bits);
        w2 = __funnelshift_l(w1, w2, bits);
        w1 = __funnelshift_l(w0, w1, bits);
        w0 <<= bits;
        const unsigned ext = (unsigned)(x >> 31);
        asm("add.cc.u32 %0, %0, %6;\n\t"
            "addc.cc.u32 %1, %1, %7;\n\t"
            "addc.cc.u32 %2, %2, %7;\n\t"
            "addc.cc.u32 %3, %3, %7;\n\t"
            "addc.cc.u32 %4, %4, %7;\n\t"
            "addc.u32 %5, %5, %7;"
            : "+r"(w0), "+r"(w1), "+r"(w2), "+r"(w3), "+r"(w4), "+r"(w5)
            : "r"((unsigned)x), "r"(ext));
    }
    unsigned long long v[3] = {((unsigned long long)w1 << 32) | w0, ((unsigned long long)w3 << 32) | w2,
                               ((unsigned long long)w5 << 32) | w4};
    bool neg = (long long)v[2] < 0;
    if (neg) neg192(v);
    const int E = e[i] + f[j] + 2 * head - bits * (S + 1);
    int p1;
    unsigned long long M1 = rn53(v, p1);
    double hi = ldexp((double)M1, p1 + E);
    // remainder r = v - M1 2^p1 (exact, may be negative)
    unsigned long long r[3] = {v[0], v[1], v[2]};
    {
        unsigned long long t[3] = {0ull, 0ull, 0ull};
        add_shifted(t, (long long)M1, p1);   // M1 <= 2^53, p1 < 128
        neg192(t);
        unsigned long long c = 0;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            unsigned long long s1 = r[q] + t[q];
            unsigned long long c1 = s1 < r[q] ? 1ull : 0ull;
            unsigned long long s2 = s1 + c;
            unsigned long long c2 = s2 < s1 ? 1ull : 0ull;
            r[q] = s2;
            c = c1 | c2;
        }
    }
    bool rneg = (long long)r[2] < 0;
    if (rneg) neg192(r);
    int p2;
    unsigned long long M2 = rn53(r, p2);
    double lo = ldexp((double)M2, p2 + E);
    if (rneg) lo = -lo;
    if (neg) {
        hi = -hi;
        lo = -lo;
    }
    C[idx] = hi;
    C[mn + idx] = lo;
}

// Step 4 rounded to T terms (QD: T = 4) on NW = 5 64-bit words:
// V = sum_g L_g 2^(bits (S + 1 - g)) by Horner's rule (|V| < 2^(32 + bits
// (S - 1)) <= 2^267), then x_t = RN(V - x_0 - ... - x_{t-1}) for t < T,
// each remainder exact, scaled by 2^(e_i + f_j + 2 head - bits (S + 1)).
template <int NW>
__device__ __forceinline__ bool wide_neg_sign(const unsigned long long (&v)[NW]) {
    return (long long)v[NW - 1] < 0;
}
template <int NW>
__device__ __forceinline__ void wide_negate(unsigned long long (&v)[NW]) {
    unsigned long long c = 1ull;
#pragma unroll
    for (int i = 0; i < NW; i++) {
        const unsigned long long x = ~v[i] + c;
        c = (c && x == 0ull) ? 1ull : 0ull;
        v[i] = x;
    }
}
template <int NW>
__device__ __forceinline__ int wide_top_bit(const unsigned long long (&v)[NW]) {
    int t = -1;
#pragma unroll
    for (int i = 0; i < NW; i++)
        if (v[i]) t = 64 * i + 63 - __clzll(v[i]);
    return t;
}
template <int NW>
__device__ __forceinline__ unsigned long long wide_bits(const unsigned long long (&v)[NW], int lo, int cnt) {
    // bits [lo, lo + cnt), cnt <= 64, lo >= 0
    const int q = lo >> 6, r = lo & 63;
    unsigned long long a = 0ull, b = 0ull;
#pragma unroll
    for (int i = 0; i < NW; i++) {
        if (i == q) a = v[i];
        if (i == q + 1) b = v[i];
    }
    const unsigned long long x = r ? ((a >> r) | (b << (64 - r))) : a;
    return cnt >= 64 ? x : (x & ((1ull << cnt) - 1ull));
}
template <int NW>
__device__ __forceinline__ bool wide_any_below(const unsigned long long (&v)[NW], int pos) {
    const int q = pos >> 6, r = pos & 63;
    bool any = false;
#pragma unroll
    for (int i = 0; i < NW; i++) {
        if (i < q) any |= v[i] != 0ull;
        if (i == q && r) any |= (v[i] & ((1ull << r) - 1ull)) != 0ull;
    }
    return any;
}

template <int T>
__global__ void k_recombine_terms(int64_t m, int64_t n, int S, int head, const int* Lv, const int* e, const int* f,
                                  double* C) {
    constexpr int NW = 5, bits = 5;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = blockIdx.y;
    if (j >= n) return;
    const int64_t mn = m * n, idx = i * n + j;
    unsigned long long v[NW];
    horner_levels<5, NW, 6>(Lv + idx, mn, S, v);
    const int E = e[i] + f[j] + 2 * head - bits * (S + 1);
#pragma unroll
    for (int t = 0; t < T; t++) {
        const bool neg = wide_neg_sign<NW>(v);
        unsigned long long a[NW];
#pragma unroll
        for (int q = 0; q < NW; q++) a[q] = v[q];
        if (neg) wide_negate<NW>(a);
        const int top = wide_top_bit<NW>(a);
        double x = 0.0;
        if (top >= 0) {
            unsigned long long M;
            int pos;
            if (top <= 52) {
                M = a[0];
                pos = 0;
            } else {
                M = wide_bits<NW>(a, top - 52, 53);
                const bool rb = wide_bits<NW>(a, top - 53, 1) != 0ull;
                const bool st = wide_any_below<NW>(a, top - 53);
                if (rb && (st || (M & 1ull))) M += 1ull;
                pos = top - 52;
            }
            x = ldexp((double)M, pos + E);
            if (neg) x = -x;
            wide_add_shifted<NW>(v, M, pos, !neg);   // v -= x (exact)
        }
        C[(int64_t)t * mn + idx] = x;
    }
}

// ---------------------------------------------------------------- driver

static size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

// K padded to 128 bytes: a whole number of K blocks for both level kernels.
int64_t ozaki_padded_k(int64_t l) { return (l + 127) / 128 * 128; }

size_t ozaki_workspace_bytes(int64_t m, int64_t l, int64_t n, int S) {
    int64_t lp = ozaki_padded_k(l);
    return a256(sizeof(int) * (size_t)m) + a256(sizeof(int) * (size_t)n) + a256((size_t)S * (size_t)(m * lp)) +
           a256((size_t)S * (size_t)(n * lp)) + a256(sizeof(int) * (size_t)S * (size_t)(m * n));
}

// Digit kinds: 0 = int8 base-128 digits (7 bits, no headroom, S <= 18),
//              1 = FP8 e4m3 balanced base-32 digits (5 bits, 1 bit headroom, S <= 24).
static int digit_bits(int kind) { return kind == 1 ? 5 : 7; }
static int digit_head(int kind) { return kind == 1 ? 1 : 0; }
static int max_slices(int kind) { return kind == 1 ? 24 : 18; }

// Column exponents of a rows x cols leading plane (0 for an all-zero column).
static int col_exponents(int64_t rows, int64_t cols, const double* X, int* expo, cudaStream_t s) {
    MPG_CUDA(cudaMemsetAsync(expo, 0x80, sizeof(int) * (size_t)cols, s));   // COLX_EMPTY
    if (rows > 0) {
        dim3 g(ceil_div(cols, 32), ceil_div(rows, COLX_ROWS));
        k_col_expo<<<g, dim3(32, 8), 0, s>>>(rows, cols, X, expo);
        if (int rc = check_launch()) return rc;
    }
    k_expo_fix<<<ceil_div(cols, 256), 256, 0, s>>>(cols, expo);
    return check_launch();
}

// FP8 digits of a T-term expansion matrix (QD: T = 4): exponents of the
// leading plane, then the balanced base-32 digits (rows: K contiguous; by
// column: transposed to K contiguous).
static int split_terms(int T, int by_col, int64_t rows, int64_t cols, const double* X, int S, int* expo, void* D,
                       int64_t lp, cudaStream_t s) {
    if (T != 4) return MPGEMM_EUNSUPPORTED;
    Bias4 C;
    b32_bias_wide<4>(S, C.w);
    if (!by_col) {
        k_row_expo<<<ceil_div(rows, 8), 256, 0, s>>>(rows, cols, X, expo);
        if (int rc = check_launch()) return rc;
        dim3 g(ceil_div(lp, 4 * 128), (unsigned)rows);
        k_slice_rows_f8_terms<4><<<g, 128, 0, s>>>(rows, cols, lp, X, expo, S, C, (unsigned char*)D);
    } else {
        if (int rc = col_exponents(rows, cols, X, expo, s)) return rc;
        const int smem = S * SLC_COLS * SLC_PITCH * 4;
        MPG_CUDA(cudaFuncSetAttribute(k_slice_cols_f8_terms<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      QD_SMAX * SLC_COLS * SLC_PITCH * 4));
        dim3 g((unsigned)(lp / SLC_ROWS), ceil_div(cols, SLC_COLS));
        k_slice_cols_f8_terms<4><<<g, 128, smem, s>>>(rows, cols, lp, X, expo, S, C, (unsigned char*)D);
    }
    return check_launch();
}

int ozaki_split(int kind, int by_col, int64_t rows, int64_t cols, const double* X, int S, int* expo, void* D,
                int64_t lp, cudaStream_t s) {
    unsigned long long Ch, Cl;
    b32_bias(S, Ch, Cl);
    if (!by_col) {
        k_row_expo<<<ceil_div(rows, 8), 256, 0, s>>>(rows, cols, X, expo);
        if (int rc = check_launch()) return rc;
        if (kind == 1) {
            const int vec = ((uintptr_t)X % 16 == 0) && (cols % 2 == 0);
            dim3 g(ceil_div(lp, 4 * 128), (unsigned)rows);
            k_slice_rows_f8<<<g, 128, 0, s>>>(rows, cols, lp, X, expo, S, Ch, Cl, vec, (unsigned char*)D);
        } else {
            dim3 g(ceil_div(lp, 128), (unsigned)rows);
            k_slice_rows<<<g, 128, 0, s>>>(rows, cols, lp, X, expo, S, (signed char*)D);
        }
    } else {
        if (int rc = col_exponents(rows, cols, X, expo, s)) return rc;
        if (kind == 1) {
            // set on every call: the current context may be an SM partition's (partition.cu)
            const int smem_max = 24 * SLC_COLS * SLC_PITCH * 4;
            MPG_CUDA(cudaFuncSetAttribute(k_slice_cols_f8, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max));
            dim3 g((unsigned)(lp / SLC_ROWS), ceil_div(cols, SLC_COLS));
            k_slice_cols_f8<<<g, 128, (size_t)S * SLC_COLS * SLC_PITCH * 4, s>>>(rows, cols, lp, X, expo, S, Ch, Cl,
                                                                               (unsigned char*)D);
        } else {
            dim3 g(ceil_div(lp, 128), (unsigned)cols);
            k_slice_cols<<<g, 128, 0, s>>>(rows, cols, lp, X, expo, S, (signed char*)D);
        }
    }
    return check_launch();
}

static int levels_launch(int64_t m, int64_t n, int64_t lp, int S, const void* DA, const void* DB, int* Lv,
                         cudaStream_t s) {
    // set on every call: the current context may be an SM partition's (partition.cu)
    MPG_CUDA(cudaFuncSetAttribute(k_ozaki_levels, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
    unsigned tm = ceil_div(m, OZ_BM), tn = ceil_div(n, OZ_BN);
    ProfScope ps(s);
    k_ozaki_levels<<<tm * tn * (unsigned)S, OZ_THREADS, OZ_SMEM, s>>>(
        m, n, lp, S, (const unsigned char*)DA, (const unsigned char*)DB, Lv, tm, tn);
    return check_launch();
}

int ozaki_levels(int kind, int64_t m, int64_t n, int64_t lp, int S, const void* DA, const void* DB, int* Lv,
                 cudaStream_t s) {
    // FP8 digits: tcgen05 (kind::f8f6f4) kernel; int8 digits: mma.sync s8 (no tcgen05 integer MMA on sm_103a)
    return kind == 1 ? tc_levels(m, n, lp, S, DA, DB, Lv, s) : levels_launch(m, n, lp, S, DA, DB, Lv, s);
}

int ozaki_recombine(int kind, int64_t m, int64_t n, int S, const int* Lv, const int* e, const int* f, double* C,
                    cudaStream_t s) {
    dim3 g(ceil_div(n, 128), (unsigned)m);
    if (digit_bits(kind) == 5) k_recombine<5><<<g, 128, 0, s>>>(m, n, S, digit_head(kind), Lv, e, f, C);
    else k_recombine<7><<<g, 128, 0, s>>>(m, n, S, digit_head(kind), Lv, e, f, C);
    return check_launch();
}

int ozaki_gemm_ws(int kind, int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int S,
                  void* ws, size_t ws_bytes, cudaStream_t s) {
    const int64_t lp = ozaki_padded_k(l);
    if (ws_bytes < ozaki_workspace_bytes(m, l, n, S)) return MPGEMM_ENOMEM;
    char* p = (char*)ws;
    int* e = (int*)p;
    p += a256(sizeof(int) * (size_t)m);
    int* f = (int*)p;
    p += a256(sizeof(int) * (size_t)n);
    void* DA = p;
    p += a256((size_t)S * (size_t)(m * lp));
    void* DB = p;
    p += a256((size_t)S * (size_t)(n * lp));
    int* Lv = (int*)p;
    int rc;
    if ((rc = ozaki_split(kind, 0, m, l, A, S, e, DA, lp, s))) return rc;
    if ((rc = ozaki_split(kind, 1, l, n, B, S, f, DB, lp, s))) return rc;
    if ((rc = ozaki_levels(kind, m, n, lp, S, DA, DB, Lv, s))) return rc;
    return ozaki_recombine(kind, m, n, S, Lv, e, f, C, s);
}

// The split-precision QD GEMM (FP8 digits, T = 4) on a caller-sized workspace.
static int ozaki_qd_gemm_ws(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int S,
                            void* ws, size_t ws_bytes, cudaStream_t s) {
    const int64_t lp = ozaki_padded_k(l);
    if (ws_bytes < ozaki_workspace_bytes(m, l, n, S)) return MPGEMM_ENOMEM;
    char* p = (char*)ws;
    int* e = (int*)p;
    p += a256(sizeof(int) * (size_t)m);
    int* f = (int*)p;
    p += a256(sizeof(int) * (size_t)n);
    void* DA = p;
    p += a256((size_t)S * (size_t)(m * lp));
    void* DB = p;
    p += a256((size_t)S * (size_t)(n * lp));
    int* Lv = (int*)p;
    int rc;
    if ((rc = split_terms(4, 0, m, l, A, S, e, DA, lp, s))) return rc;
    if ((rc = split_terms(4, 1, l, n, B, S, f, DB, lp, s))) return rc;
    if ((rc = tc_levels(m, n, lp, S, DA, DB, Lv, s))) return rc;
    dim3 g(ceil_div(n, 128), (unsigned)m);
    k_recombine_terms<4><<<g, 128, 0, s>>>(m, n, S, 1, Lv, e, f, C);
    return check_launch();
}

}  // namespace mpg

using namespace mpg;

extern "C" {

int mpgemm_qd_ozaki_slices_default(void) { return 44; }

int mpgemm_qd_ozaki(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int num_slices,
                    void* stream) {
    const int S = num_slices <= 0 ? 44 : num_slices;
    if (m < 0 || l < 0 || n < 0 || S < 1 || S > QD_SMAX) return MPGEMM_EINVAL;
    if ((m > 0 && l > 0 && !A) || (l > 0 && n > 0 && !B) || (m > 0 && n > 0 && !C)) return MPGEMM_EINVAL;
    // a slice pair's f32 sum stays below 2^24 (256 l), a level inside int32
    if (l > 65536 || (double)S * 256.0 * (double)l >= 2147483648.0) return MPGEMM_EUNSUPPORTED;
    if (m > 65535 || n > 65535) return MPGEMM_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    PartitionScope pscope(s);
    if (m == 0 || n == 0) return MPGEMM_OK;
    if (l == 0) {
        MPG_CUDA(cudaMemsetAsync(C, 0, sizeof(double) * 4 * (size_t)(m * n), s));
        return MPGEMM_OK;
    }
    size_t bytes = ozaki_workspace_bytes(m, l, n, S);
    void* ws = nullptr;
    bool owned = false;
    int rc = workspace_get(bytes, s, &ws, &owned);
    if (rc) return rc;
    rc = ozaki_qd_gemm_ws(m, l, n, A, B, C, S, ws, bytes, s);
    int rc2 = workspace_release(ws, owned, s);
    return rc ? rc : rc2;
}

int mpgemm_ozaki_split_terms(int terms, int by_col, int64_t rows, int64_t cols, const double* X, int num_slices,
                             int* expo, void* digits, void* stream) {
    if (terms != 4) return MPGEMM_EUNSUPPORTED;
    const int S = num_slices <= 0 ? 44 : num_slices;
    if (rows <= 0 || cols <= 0 || !X || !expo || !digits || S < 1 || S > QD_SMAX) return MPGEMM_EINVAL;
    if ((rows > 65535 && !by_col) || (cols > 65535 && by_col)) return MPGEMM_EUNSUPPORTED;
    PartitionScope pscope((cudaStream_t)stream);
    return split_terms(terms, by_col, rows, cols, X, S, expo, digits, ozaki_padded_k(by_col ? rows : cols),
                       (cudaStream_t)stream);
}

int mpgemm_ozaki_slices_default(void) { return 16; }

size_t mpgemm_ozaki_workspace_size(int64_t m, int64_t l, int64_t n, int num_slices) {
    if (m <= 0 || l <= 0 || n <= 0) return 0;
    int S = num_slices <= 0 ? 24 : num_slices;   // covers either digit kind's default
    return ozaki_workspace_bytes(m, l, n, S);
}

int mpgemm_dd_ozaki_ex(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int num_slices,
                       int digit_kind, void* stream) {
    if (digit_kind != 0 && digit_kind != 1) return MPGEMM_EINVAL;
    int S = num_slices <= 0 ? (digit_kind == 1 ? 22 : 16) : num_slices;
    if (m < 0 || l < 0 || n < 0 || S < 1 || S > max_slices(digit_kind)) return MPGEMM_EINVAL;
    if ((m > 0 && l > 0 && !A) || (l > 0 && n > 0 && !B) || (m > 0 && n > 0 && !C)) return MPGEMM_EINVAL;
    if (digit_kind == 0) {
        // every level sum must stay inside int32: S pairs * 127^2 * l < 2^31
        if ((double)S * 16129.0 * (double)l >= 2147483648.0) return MPGEMM_EUNSUPPORTED;
    } else {
        // a pair's f32 sum must stay below 2^24 (256 l) and a level inside int32
        if (l > 65536 || (double)S * 256.0 * (double)l >= 2147483648.0) return MPGEMM_EUNSUPPORTED;
    }
    if (m > 65535 || n > 65535) return MPGEMM_EUNSUPPORTED;   // grid.y limits of the slice kernels
    cudaStream_t s = (cudaStream_t)stream;
    PartitionScope pscope(s);
    if (m == 0 || n == 0) return MPGEMM_OK;
    if (l == 0) {
        MPG_CUDA(cudaMemsetAsync(C, 0, sizeof(double) * 2 * (size_t)(m * n), s));
        return MPGEMM_OK;
    }
    size_t bytes = ozaki_workspace_bytes(m, l, n, S);
    void* ws = nullptr;
    bool owned = false;
    int rc = workspace_get(bytes, s, &ws, &owned);
    if (rc) return rc;
    rc = ozaki_gemm_ws(digit_kind, m, l, n, A, B, C, S, ws, bytes, s);
    int rc2 = workspace_release(ws, owned, s);
    return rc ? rc : rc2;
}

int mpgemm_dd_ozaki(int64_t m, int64_t l, int64_t n, const double* A, const double* B, double* C, int num_slices,
                    void* stream) {
    return mpgemm_dd_ozaki_ex(m, l, n, A, B, C, num_slices, 0, stream);
}

int mpgemm_ozaki_split_ex(int digit_kind, int by_col, int64_t rows, int64_t cols, const double* X, int num_slices,
                          int* expo, void* digits, void* stream) {
    if (digit_kind != 0 && digit_kind != 1) return MPGEMM_EINVAL;
    int S = num_slices <= 0 ? (digit_kind == 1 ? 22 : 16) : num_slices;
    if (rows <= 0 || cols <= 0 || !X || !expo || !digits || S < 1 || S > max_slices(digit_kind)) return MPGEMM_EINVAL;
    if (rows > 65535 && !by_col) return MPGEMM_EUNSUPPORTED;
    if (cols > 65535 && by_col) return MPGEMM_EUNSUPPORTED;
    int64_t inner = by_col ? rows : cols;
    PartitionScope pscope((cudaStream_t)stream);
    return ozaki_split(digit_kind, by_col, rows, cols, X, S, expo, digits, ozaki_padded_k(inner), (cudaStream_t)stream);
}

int mpgemm_ozaki_split(int by_col, int64_t rows, int64_t cols, const double* X, int num_slices, int* expo,
                       signed char* digits, void* stream) {
    return mpgemm_ozaki_split_ex(0, by_col, rows, cols, X, num_slices, expo, digits, stream);
}

int mpgemm_ozaki_levels_ex(int digit_kind, int64_t m, int64_t l, int64_t n, int num_slices, const void* DA,
                           const void* DB, int* levels, void* stream) {
    if (digit_kind != 0 && digit_kind != 1) return MPGEMM_EINVAL;
    int S = num_slices <= 0 ? (digit_kind == 1 ? 22 : 16) : num_slices;
    if (m <= 0 || l <= 0 || n <= 0 || !DA || !DB || !levels || S < 1 || S > max_slices(digit_kind))
        return MPGEMM_EINVAL;
    if (digit_kind == 1 && l > 65536) return MPGEMM_EUNSUPPORTED;
    PartitionScope pscope((cudaStream_t)stream);
    return ozaki_levels(digit_kind, m, n, ozaki_padded_k(l), S, DA, DB, levels, (cudaStream_t)stream);
}

int mpgemm_ozaki_levels(int64_t m, int64_t l, int64_t n, int num_slices, const signed char* DA,
                        const signed char* DB, int* levels, void* stream) {
    return mpgemm_ozaki_levels_ex(0, m, l, n, num_slices, DA, DB, levels, stream);
}

}  // extern "C"
