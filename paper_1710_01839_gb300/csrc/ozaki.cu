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
#include "profile.h"
#include "strassen.h"
#include "tc_levels.h"

namespace mpg {

// ---------------------------------------------------------------- step 1

__device__ __forceinline__ int expo_of(double x) {
    if (x == 0.0) return INT_MIN;
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
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

// One thread per column, rows walked in order (coalesced across threads).
__global__ void k_col_expo(int64_t l, int64_t n, const double* hi, int* f) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int mx = INT_MIN;
    for (int64_t k = 0; k < l; k++) mx = max(mx, expo_of(hi[k * n + j]));
    f[j] = mx == INT_MIN ? 0 : mx;
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

// FP8 e4m3 code of a small integer |v| <= 16 (exact: at most 4 significant bits).
__device__ __forceinline__ unsigned char e4m3_of_int(int v) {
    unsigned s = v < 0 ? 0x80u : 0u;
    int a = v < 0 ? -v : v;
    if (a == 0) return (unsigned char)s;
    int e = 31 - __clz(a);                             // floor(log2 a), 0..4
    unsigned mant = (unsigned)((a << 3) >> e) & 7u;    // (a / 2^e - 1) * 8
    return (unsigned char)(s | ((unsigned)(e + 7) << 3) | mant);
}

// Balanced base-32 digits (FP8 variant): T = trunc((hi + lo) 2^(5S - e - 1))
// (one bit of headroom, |T| < 2^(5S-1)), written from the least significant
// digit up with digits >= 16 replaced by digit - 32 and a carry into the next
// one; the top digit keeps its carry (<= 16).  Stored as e4m3 codes.
__device__ __forceinline__ void dd_digits_b32(double hi, double lo, int e, int S, unsigned char* d, int64_t stride) {
    const int sc = 5 * S - e - 1;
    double H = ldexp(hi, sc), L = ldexp(lo, sc);
    double tH = trunc(H);
    double corr = 0.0;
    if (tH == H) {
        if (H > 0.0 && L < 0.0) corr = floor(L);
        else if (H < 0.0 && L > 0.0) corr = ceil(L);
        else corr = trunc(L);
    }
    unsigned long long th, tl, ch, cl;
    dbl_int_to_u128(tH, th, tl);
    dbl_int_to_u128(corr, ch, cl);
    bool neg;
    add_s128(th, tl, tH < 0.0, ch, cl, corr < 0.0, neg);
    int carry = 0;
    for (int s = S - 1; s >= 0; s--) {
        int sh = 5 * (S - 1 - s);
        unsigned long long v = sh >= 64 ? (th >> (sh - 64)) : (sh == 0 ? tl : ((tl >> sh) | (th << (64 - sh))));
        int dig = (int)(v & 31ull) + carry;
        carry = 0;
        if (s > 0 && dig >= 16) {
            dig -= 32;
            carry = 1;
        }
        d[(int64_t)s * stride] = e4m3_of_int(neg ? -dig : dig);
    }
}

// A (m x l, row scale e): digits into S planes of m x lp (K contiguous, zero padded).
__global__ void k_slice_rows_f8(int64_t m, int64_t l, int64_t lp, const double* A, const int* e, int S,
                                unsigned char* D) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = blockIdx.y;
    if (k >= lp || i >= m) return;
    unsigned char* out = D + i * lp + k;
    const int64_t plane = m * lp;
    if (k >= l) {
        for (int s = 0; s < S; s++) out[s * plane] = 0;
        return;
    }
    const int64_t idx = i * l + k;
    dd_digits_b32(A[idx], A[m * l + idx], e[i], S, out, plane);
}

__global__ void k_slice_cols_f8(int64_t l, int64_t n, int64_t lp, const double* B, const int* f, int S,
                                unsigned char* D) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t j = blockIdx.y;
    if (k >= lp || j >= n) return;
    unsigned char* out = D + j * lp + k;
    const int64_t plane = n * lp;
    if (k >= l) {
        for (int s = 0; s < S; s++) out[s * plane] = 0;
        return;
    }
    const int64_t idx = k * n + j;
    dd_digits_b32(B[idx], B[l * n + idx], f[j], S, out, plane);
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
// FP8 e4m3 x e4m3 -> f32: exact on the digit products (integers <= 256) as
// long as every partial sum stays below 2^24 in magnitude.
__device__ __forceinline__ void mma_e4m3(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
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
// warp tile 64 x 32 = 4 x 4 mma tiles; 4-stage cp.async pipeline.
// F8 = false: int8 digits, s32 accumulators.  F8 = true: e4m3 digit codes,
// f32 accumulators emptied into s32 after every slice pair (a pair's sum is
// at most 256 l < 2^24, so every f32 partial sum is an exact integer).
template <bool F8>
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
    float facc[F8 ? 4 : 1][F8 ? 4 : 1][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[a][b][c] = 0;
    if constexpr (F8) {
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
            for (int b = 0; b < 4; b++)
#pragma unroll
                for (int c = 0; c < 4; c++) facc[a][b][c] = 0.f;
    }

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
                for (int ni = 0; ni < 4; ni++) {
                    if constexpr (F8)
                        mma_e4m3(facc[mi][ni], a[mi], b[ni >> 1][(ni & 1) * 2], b[ni >> 1][(ni & 1) * 2 + 1]);
                    else
                        mma_s8(acc[mi][ni], a[mi], b[ni >> 1][(ni & 1) * 2], b[ni >> 1][(ni & 1) * 2 + 1]);
                }
        }
        if constexpr (F8) {
            if (it % ksteps == ksteps - 1) {   // end of a slice pair: move the exact f32 sums to s32
#pragma unroll
                for (int a = 0; a < 4; a++)
#pragma unroll
                    for (int b = 0; b < 4; b++)
#pragma unroll
                        for (int c = 0; c < 4; c++) {
                            acc[a][b][c] += __float2int_rn(facc[a][b][c]);
                            facc[a][b][c] = 0.f;
                        }
            }
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
__global__ void k_recombine(int64_t m, int64_t n, int S, int bits, int head, const int* Lv, const int* e,
                            const int* f, double* C) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = blockIdx.y;
    if (j >= n) return;
    const int64_t mn = m * n, idx = i * n + j;
    unsigned long long v[3] = {0ull, 0ull, 0ull};
    for (int g = 2; g <= S + 1; g++) add_shifted(v, (long long)Lv[(int64_t)(g - 2) * mn + idx], bits * (S + 1 - g));
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

int ozaki_split(int kind, int by_col, int64_t rows, int64_t cols, const double* X, int S, int* expo, void* D,
                int64_t lp, cudaStream_t s) {
    if (!by_col) {
        k_row_expo<<<ceil_div(rows, 8), 256, 0, s>>>(rows, cols, X, expo);
        if (int rc = check_launch()) return rc;
        dim3 g(ceil_div(lp, 128), (unsigned)rows);
        if (kind == 1) k_slice_rows_f8<<<g, 128, 0, s>>>(rows, cols, lp, X, expo, S, (unsigned char*)D);
        else k_slice_rows<<<g, 128, 0, s>>>(rows, cols, lp, X, expo, S, (signed char*)D);
    } else {
        k_col_expo<<<ceil_div(cols, 128), 128, 0, s>>>(rows, cols, X, expo);
        if (int rc = check_launch()) return rc;
        dim3 g(ceil_div(lp, 128), (unsigned)cols);
        if (kind == 1) k_slice_cols_f8<<<g, 128, 0, s>>>(rows, cols, lp, X, expo, S, (unsigned char*)D);
        else k_slice_cols<<<g, 128, 0, s>>>(rows, cols, lp, X, expo, S, (signed char*)D);
    }
    return check_launch();
}

template <bool F8>
static int levels_launch(int64_t m, int64_t n, int64_t lp, int S, const void* DA, const void* DB, int* Lv,
                         cudaStream_t s) {
    static bool attr_set[64];
    int dev = 0;
    MPG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return MPGEMM_EUNSUPPORTED;
    if (!attr_set[dev]) {
        MPG_CUDA(cudaFuncSetAttribute(k_ozaki_levels<F8>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM));
        attr_set[dev] = true;
    }
    unsigned tm = ceil_div(m, OZ_BM), tn = ceil_div(n, OZ_BN);
    ProfScope ps(s);
    k_ozaki_levels<F8><<<tm * tn * (unsigned)S, OZ_THREADS, OZ_SMEM, s>>>(
        m, n, lp, S, (const unsigned char*)DA, (const unsigned char*)DB, Lv, tm, tn);
    return check_launch();
}

int ozaki_levels(int kind, int64_t m, int64_t n, int64_t lp, int S, const void* DA, const void* DB, int* Lv,
                 cudaStream_t s) {
    // FP8 digits: tcgen05 (kind::f8f6f4) kernel; int8 digits: mma.sync s8 (no tcgen05 integer MMA on sm_103a)
    return kind == 1 ? tc_levels(m, n, lp, S, DA, DB, Lv, s) : levels_launch<false>(m, n, lp, S, DA, DB, Lv, s);
}

int ozaki_recombine(int kind, int64_t m, int64_t n, int S, const int* Lv, const int* e, const int* f, double* C,
                    cudaStream_t s) {
    dim3 g(ceil_div(n, 128), (unsigned)m);
    k_recombine<<<g, 128, 0, s>>>(m, n, S, digit_bits(kind), digit_head(kind), Lv, e, f, C);
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

}  // namespace mpg

using namespace mpg;

extern "C" {

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
    if ((m * l && !A) || (l * n && !B) || (m * n && !C)) return MPGEMM_EINVAL;
    if (digit_kind == 0) {
        // every level sum must stay inside int32: S pairs * 127^2 * l < 2^31
        if ((double)S * 16129.0 * (double)l >= 2147483648.0) return MPGEMM_EUNSUPPORTED;
    } else {
        // a pair's f32 sum must stay below 2^24 (256 l) and a level inside int32
        if (l > 65536 || (double)S * 256.0 * (double)l >= 2147483648.0) return MPGEMM_EUNSUPPORTED;
    }
    if (m > 65535 || n > 65535) return MPGEMM_EUNSUPPORTED;   // grid.y limits of the slice kernels
    cudaStream_t s = (cudaStream_t)stream;
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
    return ozaki_levels(digit_kind, m, n, ozaki_padded_k(l), S, DA, DB, levels, (cudaStream_t)stream);
}

int mpgemm_ozaki_levels(int64_t m, int64_t l, int64_t n, int num_slices, const signed char* DA,
                        const signed char* DB, int* levels, void* stream) {
    return mpgemm_ozaki_levels_ex(0, m, l, n, num_slices, DA, DB, levels, stream);
}

}  // extern "C"
