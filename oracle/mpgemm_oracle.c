/*
 * ORACLE — plain, slow CPU reference for multiple-precision dense real GEMM
 * C := AB (A m x l, B l x n), after Kouya, "Tuning Technique for Multiple
 * Precision Dense Matrix Multiplication using Prediction of Computational
 * Time" (arXiv:1710.01839), Section 2, Eqs 1-3.
 *
 * This file is TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it.  The CUDA library never calls
 * it, shares no code, header or table with it, and must not fall back to it.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC.
 * Contraction must stay off: every FMA below is an explicit fma() call, named
 * by the algorithm it belongs to; every other product and sum is a separately
 * rounded IEEE-754 binary64 operation.
 *
 * Contents (each function cites what it follows):
 *   - error-free transformations (TwoSum, Fast2Sum, TwoProd)
 *   - double-double (DD) add and multiply
 *   - an exact wide fixed-point accumulator (used for quad-double rounding and
 *     as the exact checker of sampled GEMM entries)
 *   - quad-double (QD): every operation is "exact result, rounded to four
 *     non-overlapping doubles by greedy round-to-nearest extraction"
 *   - p-bit multi-limb binary floats (p = 32 w), round-to-nearest-even per op
 *   - the three GEMM algorithms (simple Eq 1, block Eq 2, Strassen Eq 3) over
 *     any of the three formats
 *   - the split-precision (Ozaki-style) DD GEMM steps: exponent extraction,
 *     int8 digit slicing, exact integer slice products, recombination
 *
 * Matrix layout at the ABI: row-major "planes".  A DD matrix is two
 * contiguous m*l double arrays [hi | lo]; QD has four planes x0..x3; a
 * multi-limb matrix is (2 + w) uint32 planes: [exponent (int32) | flags |
 * limb 0 (least significant) ... limb w-1 (most significant)].  A multi-limb
 * value is (-1)^s * M * 2^(e - p) with M in [2^(p-1), 2^p) (MPFR's 0.M * 2^e
 * convention); flags bit0 = sign, bit1 = zero (M = 0, e = 0).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_API __attribute__((visibility("default")))

static int g_threads = 0; /* 0: OpenMP default */

OR_API void or_set_threads(int t) { g_threads = t; }
OR_API int or_get_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

static void die(const char *msg) {
    fprintf(stderr, "oracle: %s\n", msg);
    abort();
}

/* ------------------------------------------------------------------------ */
/* Error-free transformations                                                */
/* ------------------------------------------------------------------------ */

/* Knuth's TwoSum: s = RN(a+b), e = (a+b) - s exactly, no precondition. */
static inline void two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    double br = b - bv;
    double ar = a - av;
    *s = x;
    *e = ar + br;
}

/* Dekker's Fast2Sum: exact when exponent(a) >= exponent(b) (or a == 0). */
static inline void fast_two_sum(double a, double b, double *s, double *e) {
    double x = a + b;
    double z = x - a;
    *s = x;
    *e = b - z;
}

/* TwoProd with one FMA: p = RN(ab), e = ab - p exactly (no underflow). */
static inline void two_prod(double a, double b, double *p, double *e) {
    double x = a * b;
    *p = x;
    *e = fma(a, b, -x);
}

OR_API void or_two_sum(double a, double b, double *out) { two_sum(a, b, &out[0], &out[1]); }
OR_API void or_fast_two_sum(double a, double b, double *out) { fast_two_sum(a, b, &out[0], &out[1]); }
OR_API void or_two_prod(double a, double b, double *out) { two_prod(a, b, &out[0], &out[1]); }

/* ------------------------------------------------------------------------ */
/* Double-double (the DD type of the QD library the paper uses, Section 1).  */
/* The paper does not print the DD algorithms; the oracle uses the           */
/* double-word algorithms of Joldes, Muller & Popescu, "Tight and rigorous   */
/* error bounds for basic building blocks of double-word arithmetic" (2017). */
/* ------------------------------------------------------------------------ */

typedef struct { double hi, lo; } dd_t;

/* Accurate double-word + double-word (relative error <= 3u^2 + O(u^3)). */
static inline dd_t dd_add(dd_t x, dd_t y) {
    double sh, sl, th, tl, c, vh, vl, w;
    dd_t z;
    two_sum(x.hi, y.hi, &sh, &sl);
    two_sum(x.lo, y.lo, &th, &tl);
    c = sl + th;
    fast_two_sum(sh, c, &vh, &vl);
    w = tl + vl;
    fast_two_sum(vh, w, &z.hi, &z.lo);
    return z;
}

static inline dd_t dd_neg(dd_t x) { dd_t z = {-x.hi, -x.lo}; return z; }
static inline dd_t dd_sub(dd_t x, dd_t y) { return dd_add(x, dd_neg(y)); }

/* Double-word x double-word with FMA, the variant that also forms xl*yl
   (relative error <= 5u^2). */
static inline dd_t dd_mul(dd_t x, dd_t y) {
    double ch, cl1, tl0, tl1, cl2, cl3;
    dd_t z;
    two_prod(x.hi, y.hi, &ch, &cl1);
    tl0 = x.lo * y.lo;
    tl1 = fma(x.hi, y.lo, tl0);
    cl2 = fma(x.lo, y.hi, tl1);
    cl3 = cl1 + cl2;
    fast_two_sum(ch, cl3, &z.hi, &z.lo);
    return z;
}

OR_API void or_dd_add(const double *x, const double *y, double *z) {
    dd_t a = {x[0], x[1]}, b = {y[0], y[1]}, c = dd_add(a, b);
    z[0] = c.hi; z[1] = c.lo;
}
OR_API void or_dd_mul(const double *x, const double *y, double *z) {
    dd_t a = {x[0], x[1]}, b = {y[0], y[1]}, c = dd_mul(a, b);
    z[0] = c.hi; z[1] = c.lo;
}

/* ------------------------------------------------------------------------ */
/* Exact wide fixed-point accumulator.                                       */
/* Two's complement over WFX_LIMBS 32-bit limbs; bit i has weight            */
/* 2^(i - WFX_FRAC).  Range (-2^191, 2^191), resolution 2^-1216: enough for   */
/* every exact product and sum of the formats at the magnitudes used here.   */
/* Anything outside the window aborts loudly.                                */
/* ------------------------------------------------------------------------ */

#define WFX_LIMBS 44
#define WFX_FRAC 1216

typedef struct { uint32_t w[WFX_LIMBS]; } wfx_t;

static inline void wfx_zero(wfx_t *a) { memset(a->w, 0, sizeof a->w); }

/* a += (neg ? -1 : 1) * m * 2^pos, pos = bit index in the window. */
static void wfx_addsub(wfx_t *a, uint64_t m, int pos, int neg) {
    unsigned __int128 v;
    uint32_t ch[3];
    int li, sh, t, idx;
    if (m == 0) return;
    if (pos < 0) {
        if (pos <= -64 || (m & ((1ULL << (-pos)) - 1ULL)) != 0) die("exact accumulator underflow");
        m >>= (-pos);
        pos = 0;
    }
    li = pos >> 5;
    sh = pos & 31;
    v = ((unsigned __int128)m) << sh;
    ch[0] = (uint32_t)v;
    ch[1] = (uint32_t)(v >> 32);
    ch[2] = (uint32_t)(v >> 64);
    if (!neg) {
        uint64_t carry = 0;
        for (t = 0; t < 3; t++) {
            idx = li + t;
            if (idx >= WFX_LIMBS) { if (ch[t] || carry) die("exact accumulator overflow"); continue; }
            uint64_t s = (uint64_t)a->w[idx] + ch[t] + carry;
            a->w[idx] = (uint32_t)s;
            carry = s >> 32;
        }
        for (idx = li + 3; carry && idx < WFX_LIMBS; idx++) {
            uint64_t s = (uint64_t)a->w[idx] + carry;
            a->w[idx] = (uint32_t)s;
            carry = s >> 32;
        }
    } else {
        uint64_t borrow = 0;
        for (t = 0; t < 3; t++) {
            idx = li + t;
            if (idx >= WFX_LIMBS) { if (ch[t] || borrow) die("exact accumulator overflow"); continue; }
            uint64_t sub = (uint64_t)ch[t] + borrow;
            uint64_t cur = a->w[idx];
            a->w[idx] = (uint32_t)(cur - sub);
            borrow = cur < sub;
        }
        for (idx = li + 3; borrow && idx < WFX_LIMBS; idx++) {
            uint64_t cur = a->w[idx];
            a->w[idx] = (uint32_t)(cur - 1);
            borrow = (cur == 0);
        }
    }
}

/* a += x exactly. */
static void wfx_add_double(wfx_t *a, double x) {
    int e;
    double f;
    uint64_t m;
    if (x == 0.0) return;
    if (!isfinite(x)) die("non-finite value");
    f = frexp(fabs(x), &e);           /* |x| = f * 2^e, f in [0.5, 1) */
    m = (uint64_t)ldexp(f, 53);       /* exact 53-bit integer */
    wfx_addsub(a, m, e - 53 + WFX_FRAC, x < 0);
}

/* a += x*y exactly (TwoProd; no underflow at the magnitudes used). */
static void wfx_add_prod(wfx_t *a, double x, double y) {
    double p, e;
    two_prod(x, y, &p, &e);
    wfx_add_double(a, p);
    wfx_add_double(a, e);
}

static inline int wfx_is_neg(const wfx_t *a) { return (a->w[WFX_LIMBS - 1] >> 31) & 1; }

static void wfx_negate(wfx_t *a) {
    uint64_t carry = 1;
    for (int i = 0; i < WFX_LIMBS; i++) {
        uint64_t s = (uint64_t)(uint32_t)~a->w[i] + carry;
        a->w[i] = (uint32_t)s;
        carry = s >> 32;
    }
}

/* Bits [lo, lo + cnt) of the window, cnt <= 53. */
static uint64_t wfx_bits(const wfx_t *a, int lo, int cnt) {
    unsigned __int128 x = 0;
    int q = lo >> 5, r = lo & 31;
    for (int t = 2; t >= 0; t--) {
        int idx = q + t;
        x <<= 32;
        if (idx >= 0 && idx < WFX_LIMBS) x |= a->w[idx];
    }
    return (uint64_t)(x >> r) & ((1ULL << cnt) - 1ULL);
}

/* Is any bit below position i set? */
static int wfx_any_below(const wfx_t *a, int i) {
    int q = i >> 5, r = i & 31;
    for (int t = 0; t < q && t < WFX_LIMBS; t++)
        if (a->w[t]) return 1;
    if (r && q < WFX_LIMBS && (a->w[q] & ((1u << r) - 1u))) return 1;
    return 0;
}

/* Round the exact value to the nearest double, ties to even. */
static double wfx_round(const wfx_t *src) {
    wfx_t a = *src;
    int neg = wfx_is_neg(&a), top = -1, i;
    uint64_t mant;
    int rbit, sticky;
    double r;
    if (neg) wfx_negate(&a);
    for (i = WFX_LIMBS - 1; i >= 0; i--) {
        if (a.w[i]) { top = i * 32 + 31 - __builtin_clz(a.w[i]); break; }
    }
    if (top < 0) return 0.0;
    if (top - WFX_FRAC < -1022) die("exact accumulator result below the normal range");
    if (top <= 53) die("exact accumulator result too small");
    mant = wfx_bits(&a, top - 52, 53);
    rbit = (int)wfx_bits(&a, top - 53, 1);
    sticky = wfx_any_below(&a, top - 53);
    if (rbit && (sticky || (mant & 1))) mant += 1;
    r = ldexp((double)mant, top - 52 - WFX_FRAC);
    return neg ? -r : r;
}

/* Greedy extraction: x[t] = RN(a - x[0] - ... - x[t-1]), t < nterms. */
static void wfx_round_terms(wfx_t *a, double *x, int nterms) {
    for (int t = 0; t < nterms; t++) {
        x[t] = wfx_round(a);
        wfx_add_double(a, -x[t]);
    }
}

/* ------------------------------------------------------------------------ */
/* Quad-double (the QD type of the QD library, Section 1).  Reading: each    */
/* QD operation returns its exact result rounded to four non-overlapping     */
/* doubles by greedy round-to-nearest extraction (the ideal that the QD      */
/* library's add and multiply approximate).                                  */
/* ------------------------------------------------------------------------ */

typedef struct { double x[4]; } qd_t;

static qd_t qd_add(qd_t a, qd_t b) {
    wfx_t W;
    qd_t z;
    wfx_zero(&W);
    for (int i = 0; i < 4; i++) { wfx_add_double(&W, a.x[i]); wfx_add_double(&W, b.x[i]); }
    wfx_round_terms(&W, z.x, 4);
    return z;
}

static qd_t qd_neg(qd_t a) { for (int i = 0; i < 4; i++) a.x[i] = -a.x[i]; return a; }

static qd_t qd_mul(qd_t a, qd_t b) {
    wfx_t W;
    qd_t z;
    wfx_zero(&W);
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) wfx_add_prod(&W, a.x[i], b.x[j]);
    wfx_round_terms(&W, z.x, 4);
    return z;
}

OR_API void or_qd_add(const double *x, const double *y, double *z) {
    qd_t a, b, c;
    memcpy(a.x, x, sizeof a.x); memcpy(b.x, y, sizeof b.x);
    c = qd_add(a, b);
    memcpy(z, c.x, sizeof c.x);
}
OR_API void or_qd_mul(const double *x, const double *y, double *z) {
    qd_t a, b, c;
    memcpy(a.x, x, sizeof a.x); memcpy(b.x, y, sizeof b.x);
    c = qd_mul(a, b);
    memcpy(z, c.x, sizeof c.x);
}
/* Exact sum of n doubles rounded to `terms` greedy terms (pins use this). */
OR_API void or_round_terms(const double *v, int n, double *out, int terms) {
    wfx_t W;
    wfx_zero(&W);
    for (int i = 0; i < n; i++) wfx_add_double(&W, v[i]);
    wfx_round_terms(&W, out, terms);
}

/* ------------------------------------------------------------------------ */
/* p-bit multi-limb binary floats, p = 32 w (the fixed-precision stand-in    */
/* for MPFR, Section 4.2).  Every operation is rounded to nearest, ties to   */
/* even; multiply then add, two roundings per multiply-accumulate.           */
/* ------------------------------------------------------------------------ */

#define MP_WMAX 64

typedef struct {
    int64_t e;               /* value = (-1)^s * M * 2^(e - p)              */
    int s, z;                /* sign, zero flag                             */
    uint32_t m[MP_WMAX];     /* M, limb 0 least significant, M in [2^(p-1),2^p) */
} mp_t;

static int bi_bitlen(const uint32_t *a, int n) {
    for (int i = n - 1; i >= 0; i--)
        if (a[i]) return i * 32 + 32 - __builtin_clz(a[i]);
    return 0;
}
static inline int bi_bit(const uint32_t *a, int n, int64_t i) {
    if (i < 0 || i >= (int64_t)n * 32) return 0;
    return (a[i >> 5] >> (i & 31)) & 1;
}
static int bi_any_below(const uint32_t *a, int n, int64_t i) {   /* any bit < i */
    int64_t q = i >> 5;
    int r = (int)(i & 31);
    for (int64_t t = 0; t < q && t < n; t++)
        if (a[t]) return 1;
    if (r && q < n && (a[q] & ((1u << r) - 1u))) return 1;
    return 0;
}
static inline uint64_t bi_word(const uint32_t *a, int n, int64_t idx) {
    return (idx >= 0 && idx < n) ? a[idx] : 0;
}
/* dst[0..dn) = src >> sh, sh >= 0 (bits shifted out are dropped). */
static void bi_shr(uint32_t *dst, int dn, const uint32_t *src, int sn, int64_t sh) {
    int64_t q = sh >> 5;
    int r = (int)(sh & 31);
    for (int i = 0; i < dn; i++) {
        uint64_t two = (bi_word(src, sn, i + q + 1) << 32) | bi_word(src, sn, i + q);
        dst[i] = (uint32_t)(two >> r);
    }
}
/* dst[0..dn) = src << sh, sh >= 0 (bits beyond dn limbs are dropped). */
static void bi_shl(uint32_t *dst, int dn, const uint32_t *src, int sn, int64_t sh) {
    int64_t q = sh >> 5;
    int r = (int)(sh & 31);
    for (int i = 0; i < dn; i++) {
        uint64_t two = (bi_word(src, sn, i - q) << 32) | bi_word(src, sn, i - q - 1);
        dst[i] = (uint32_t)((two << r) >> 32);
    }
}
static int bi_cmp(const uint32_t *a, const uint32_t *b, int n) {
    for (int i = n - 1; i >= 0; i--) {
        if (a[i] != b[i]) return a[i] > b[i] ? 1 : -1;
    }
    return 0;
}
static void bi_add(uint32_t *d, const uint32_t *a, const uint32_t *b, int n) {
    uint64_t c = 0;
    for (int i = 0; i < n; i++) { uint64_t s = (uint64_t)a[i] + b[i] + c; d[i] = (uint32_t)s; c = s >> 32; }
    if (c) die("multi-limb add overflow");
}
static void bi_sub(uint32_t *d, const uint32_t *a, const uint32_t *b, int n) {   /* a >= b */
    uint64_t br = 0;
    for (int i = 0; i < n; i++) {
        uint64_t sub = (uint64_t)b[i] + br;
        d[i] = (uint32_t)((uint64_t)a[i] - sub);
        br = (uint64_t)a[i] < sub;
    }
    if (br) die("multi-limb subtract underflow");
}

/* Round the (sn-limb) integer S to p bits: returns M (w limbs) and the
   shift k such that S ~= M * 2^k; *carry set when rounding reached 2^p
   (M is then renormalised to 2^(p-1) and k incremented). */
static void mp_round_int(const uint32_t *S, int sn, int w, uint32_t *M, int64_t *k) {
    int p = 32 * w;
    int L = bi_bitlen(S, sn);
    if (L <= p) {
        bi_shl(M, w, S, sn, p - L);
        *k = L - p;
        return;
    }
    int64_t sh = L - p;
    bi_shr(M, w, S, sn, sh);
    int rbit = bi_bit(S, sn, sh - 1);
    int sticky = bi_any_below(S, sn, sh - 1);
    *k = sh;
    if (rbit && (sticky || (M[0] & 1))) {
        uint64_t c = 1;
        for (int i = 0; i < w && c; i++) { uint64_t s = (uint64_t)M[i] + c; M[i] = (uint32_t)s; c = s >> 32; }
        if (c) {   /* M overflowed to 2^p: M = 2^(p-1), one more power of two */
            memset(M, 0, sizeof(uint32_t) * w);
            M[w - 1] = 0x80000000u;
            *k += 1;
        }
    }
}

static mp_t mp_zero(int s) { mp_t r; memset(&r, 0, sizeof r); r.z = 1; r.s = s; return r; }

/* RN_p(x * y). */
static mp_t mp_mul(const mp_t *x, const mp_t *y, int w) {
    uint32_t P[2 * MP_WMAX];
    mp_t r;
    int64_t k;
    if (x->z || y->z) return mp_zero(x->s ^ y->s);
    memset(P, 0, sizeof(uint32_t) * 2 * w);
    for (int i = 0; i < w; i++) {          /* schoolbook, exact 2p-bit product */
        uint64_t c = 0;
        for (int j = 0; j < w; j++) {
            uint64_t t = (uint64_t)x->m[i] * y->m[j] + P[i + j] + c;
            P[i + j] = (uint32_t)t;
            c = t >> 32;
        }
        P[i + w] = (uint32_t)c;
    }
    memset(&r, 0, sizeof r);
    mp_round_int(P, 2 * w, w, r.m, &k);
    /* x*y = P * 2^(ex+ey-2p) = M * 2^k * 2^(ex+ey-2p) = M * 2^(e-p) */
    r.e = x->e + y->e - 32 * w + k;
    r.s = x->s ^ y->s;
    r.z = 0;
    return r;
}

/* RN_p(x + y). */
static mp_t mp_add(const mp_t *xin, const mp_t *yin, int w) {
    const mp_t *x = xin, *y = yin;
    uint32_t X[2 * MP_WMAX + 2], Y[2 * MP_WMAX + 2], S[2 * MP_WMAX + 2];
    int n = 2 * w + 2, p = 32 * w, sign;
    int64_t d, k;
    mp_t r;
    if (x->z && y->z) return mp_zero(x->s & y->s);
    if (x->z) return *y;
    if (y->z) return *x;
    if (x->e < y->e) { const mp_t *t = x; x = y; y = t; }
    d = x->e - y->e;
    if (d >= p + 2) return *x;           /* |y| < half an ulp of every neighbour of x */
    bi_shl(X, n, x->m, w, d);            /* exact: S = Mx*2^d +- My, value S*2^(ey-p) */
    bi_shl(Y, n, y->m, w, 0);
    if (x->s == y->s) {
        bi_add(S, X, Y, n);
        sign = x->s;
    } else {
        int c = bi_cmp(X, Y, n);
        if (c == 0) return mp_zero(0);   /* exact cancellation gives +0 */
        if (c > 0) { bi_sub(S, X, Y, n); sign = x->s; }
        else { bi_sub(S, Y, X, n); sign = y->s; }
    }
    memset(&r, 0, sizeof r);
    mp_round_int(S, n, w, r.m, &k);
    r.e = y->e + k;
    r.s = sign;
    r.z = 0;
    return r;
}

static mp_t mp_neg(mp_t x) { x.s ^= 1; return x; }

/* AoS word layout of one element inside the oracle: [e, flags, m0..m(w-1)]. */
static void mp_load(mp_t *r, const uint32_t *src, int w) {
    memset(r, 0, sizeof *r);
    r->e = (int32_t)src[0];
    r->s = src[1] & 1;
    r->z = (src[1] >> 1) & 1;
    if (!r->z) {
        memcpy(r->m, src + 2, sizeof(uint32_t) * w);
        if (!(r->m[w - 1] & 0x80000000u)) die("multi-limb input not normalised");
    }
}
static void mp_store(uint32_t *dst, const mp_t *r, int w) {
    if (r->z) {
        memset(dst, 0, sizeof(uint32_t) * (2 + w));
        dst[1] = (uint32_t)(r->s & 1) | 2u;
        return;
    }
    if (r->e > INT32_MAX || r->e < INT32_MIN) die("multi-limb exponent overflow");
    dst[0] = (uint32_t)(int32_t)r->e;
    dst[1] = (uint32_t)(r->s & 1);
    memcpy(dst + 2, r->m, sizeof(uint32_t) * w);
}

OR_API void or_mp_mul(int w, const uint32_t *x, const uint32_t *y, uint32_t *z) {
    mp_t a, b, c;
    mp_load(&a, x, w); mp_load(&b, y, w);
    c = mp_mul(&a, &b, w);
    mp_store(z, &c, w);
}
OR_API void or_mp_add(int w, const uint32_t *x, const uint32_t *y, uint32_t *z) {
    mp_t a, b, c;
    mp_load(&a, x, w); mp_load(&b, y, w);
    c = mp_add(&a, &b, w);
    mp_store(z, &c, w);
}

/* ------------------------------------------------------------------------ */
/* Conversions between T-term double expansions (DD: T = 2, QD: T = 4) and  */
/* p-bit multi-limb numbers, for the DD / QD GEMM computed in multi-limb     */
/* arithmetic (an extension of Section 2's GEMM, not in the paper):          */
/*   to p bits:   c = +0, then c = RN_p(c + x_t) for t = 0..T-1, each double */
/*                x_t taken exactly (p >= 64 bits hold its 53);              */
/*   from p bits: for t = 0..T-1: x_t = RN_53(r) (nearest double, ties to    */
/*                even), r = r - x_t (exact): the greedy expansion of c.     */
/* ------------------------------------------------------------------------ */

/* The double x exactly as a w-limb value, w >= 2. */
static mp_t mp_of_double(double x, int w) {
    mp_t r;
    int ex;
    if (!isfinite(x)) die("conversion of a non-finite double");
    if (x == 0.0) return mp_zero(signbit(x) ? 1 : 0);
    double f = frexp(fabs(x), &ex);                 /* |x| = f 2^ex, f in [1/2, 1) */
    uint64_t top = (uint64_t)ldexp(f, 64);          /* f 2^64: an integer below 2^64 */
    memset(&r, 0, sizeof r);
    r.m[w - 1] = (uint32_t)(top >> 32);             /* M = top 2^(p - 64) */
    r.m[w - 2] = (uint32_t)top;
    r.e = ex;                                       /* |x| = M 2^(ex - p) */
    r.s = signbit(x) ? 1 : 0;
    r.z = 0;
    return r;
}

/* RN_53 of a w-limb value as a double (the result must be a normal double). */
static double mp_round_double(const mp_t *v, int w) {
    if (v->z) return v->s ? -0.0 : 0.0;
    int p = 32 * w;
    uint64_t top = ((uint64_t)v->m[w - 1] << 32) | v->m[w - 2];    /* M >> (p - 64) */
    uint64_t q = top >> 11;                                         /* M >> (p - 53), 53 bits */
    int rbit = (int)((top >> 10) & 1);
    int sticky = (top & 0x3FFu) != 0 || bi_any_below(v->m, w, (int64_t)p - 64);
    if (rbit && (sticky || (q & 1))) q += 1;                        /* q in [2^52, 2^53] */
    int64_t e = v->e - 53;                                          /* value = q 2^e */
    int64_t lead = e + (q >> 53 ? 53 : 52);                         /* exponent of the leading bit */
    if (lead < -1022 || lead > 1023) die("conversion to double outside the normal range");
    double d = ldexp((double)q, (int)e);
    return v->s ? -d : d;
}

OR_API void or_terms_to_mp(int T, int64_t count, const double *X, int w, uint32_t *Y) {
    uint32_t tmp[2 + MP_WMAX];
    if (w < 2 || w > MP_WMAX) die("conversion width");
    for (int64_t i = 0; i < count; i++) {
        mp_t c = mp_zero(0);
        for (int t = 0; t < T; t++) {
            mp_t x = mp_of_double(X[t * count + i], w);
            c = mp_add(&c, &x, w);
        }
        mp_store(tmp, &c, w);
        for (int q = 0; q < 2 + w; q++) Y[q * count + i] = tmp[q];
    }
}

OR_API void or_mp_to_terms(int T, int64_t count, int w, const uint32_t *Y, double *X) {
    uint32_t tmp[2 + MP_WMAX];
    if (w < 2 || w > MP_WMAX) die("conversion width");
    for (int64_t i = 0; i < count; i++) {
        mp_t r;
        for (int q = 0; q < 2 + w; q++) tmp[q] = Y[q * count + i];
        mp_load(&r, tmp, w);
        for (int t = 0; t < T; t++) {
            double d = mp_round_double(&r, w);
            X[t * count + i] = d;
            mp_t x = mp_of_double(-d, w);
            r = mp_add(&r, &x, w);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Format-generic element operations for the GEMM algorithms.               */
/* Elements live in AoS buffers of `esz` bytes inside the oracle.           */
/* ------------------------------------------------------------------------ */

enum { F_DD = 0, F_QD = 1, F_MP = 2 };

typedef struct {
    int kind;
    int w;        /* limbs for F_MP */
    size_t esz;   /* bytes per AoS element */
} fmt_t;

static void el_zero(const fmt_t *f, void *c) {
    memset(c, 0, f->esz);
    if (f->kind == F_MP) ((uint32_t *)c)[1] = 2u;   /* +0 */
}

/* c = c + a*b (one multiply, one add, each rounded in the format). */
static void el_mac(const fmt_t *f, void *c, const void *a, const void *b) {
    if (f->kind == F_DD) {
        dd_t *C = (dd_t *)c;
        *C = dd_add(*C, dd_mul(*(const dd_t *)a, *(const dd_t *)b));
    } else if (f->kind == F_QD) {
        qd_t *C = (qd_t *)c;
        *C = qd_add(*C, qd_mul(*(const qd_t *)a, *(const qd_t *)b));
    } else {
        mp_t A, B, C, t;
        mp_load(&A, (const uint32_t *)a, f->w);
        mp_load(&B, (const uint32_t *)b, f->w);
        mp_load(&C, (const uint32_t *)c, f->w);
        t = mp_mul(&A, &B, f->w);
        C = mp_add(&C, &t, f->w);
        mp_store((uint32_t *)c, &C, f->w);
    }
}

/* z = x + y (sub: x - y), rounded in the format. */
static void el_addsub(const fmt_t *f, void *z, const void *x, const void *y, int sub) {
    if (f->kind == F_DD) {
        dd_t Y = *(const dd_t *)y;
        *(dd_t *)z = dd_add(*(const dd_t *)x, sub ? dd_neg(Y) : Y);
    } else if (f->kind == F_QD) {
        qd_t Y = *(const qd_t *)y;
        *(qd_t *)z = qd_add(*(const qd_t *)x, sub ? qd_neg(Y) : Y);
    } else {
        mp_t X, Y, Z;
        mp_load(&X, (const uint32_t *)x, f->w);
        mp_load(&Y, (const uint32_t *)y, f->w);
        if (sub) Y = mp_neg(Y);
        Z = mp_add(&X, &Y, f->w);
        mp_store((uint32_t *)z, &Z, f->w);
    }
}

/* A matrix view: element (i, j) at base + (i*ld + j)*esz. */
typedef struct { char *p; int64_t ld; } view_t;

static inline char *at(const fmt_t *f, view_t v, int64_t i, int64_t j) {
    return v.p + ((size_t)(i * v.ld + j)) * f->esz;
}

/* Eq 1, simple triple loop, rows [r0, r1) of C only: c_ij = sum_k a_ik b_kj,
   k = 1..l in ascending order, starting from zero. */
static void gemm_simple(const fmt_t *f, int64_t m, int64_t l, int64_t n, view_t A, view_t B, view_t C,
                        int64_t r0, int64_t r1) {
    (void)m;
#pragma omp parallel for schedule(dynamic, 1) num_threads(or_get_threads())
    for (int64_t i = r0; i < r1; i++) {
        for (int64_t j = 0; j < n; j++) {
            char *c = at(f, C, i, j);
            el_zero(f, c);
            for (int64_t k = 0; k < l; k++) el_mac(f, c, at(f, A, i, k), at(f, B, k, j));
        }
    }
}

/* Eq 2, block algorithm with block size n_min: C_IJ = sum_K A_IK B_KJ over
   n_min x n_min blocks, each C block accumulated in place over K blocks in
   ascending order (so every c_ij sees the same operation sequence as Eq 1).
   Rows [r0, r1) of C only; ragged edge blocks are smaller. */
static void gemm_block(const fmt_t *f, int64_t m, int64_t l, int64_t n, view_t A, view_t B, view_t C,
                       int64_t n_min, int64_t r0, int64_t r1) {
    (void)m;
    int64_t nb_i = (r1 - r0 + n_min - 1) / n_min;
    int64_t nb_j = (n + n_min - 1) / n_min;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) num_threads(or_get_threads())
    for (int64_t bi = 0; bi < nb_i; bi++) {
        for (int64_t bj = 0; bj < nb_j; bj++) {
            int64_t i0 = r0 + bi * n_min, i1 = i0 + n_min < r1 ? i0 + n_min : r1;
            int64_t j0 = bj * n_min, j1 = j0 + n_min < n ? j0 + n_min : n;
            for (int64_t i = i0; i < i1; i++)
                for (int64_t j = j0; j < j1; j++) el_zero(f, at(f, C, i, j));
            for (int64_t k0 = 0; k0 < l; k0 += n_min) {
                int64_t k1 = k0 + n_min < l ? k0 + n_min : l;
                for (int64_t i = i0; i < i1; i++)
                    for (int64_t j = j0; j < j1; j++) {
                        char *c = at(f, C, i, j);
                        for (int64_t k = k0; k < k1; k++) el_mac(f, c, at(f, A, i, k), at(f, B, k, j));
                    }
            }
        }
    }
}

/* Z = X +/- Y elementwise over an r x c view. */
static void mat_addsub(const fmt_t *f, int64_t r, int64_t c, view_t Z, view_t X, view_t Y, int sub) {
#pragma omp parallel for schedule(static) num_threads(or_get_threads())
    for (int64_t i = 0; i < r; i++)
        for (int64_t j = 0; j < c; j++) el_addsub(f, at(f, Z, i, j), at(f, X, i, j), at(f, Y, i, j), sub);
}

static view_t sub_view(const fmt_t *f, view_t v, int64_t i, int64_t j) {
    view_t r = {at(f, v, i, j), v.ld};
    return r;
}

static view_t new_mat(const fmt_t *f, int64_t r, int64_t c) {
    view_t v;
    v.p = (char *)malloc((size_t)(r * c) * f->esz + 1);
    if (!v.p) die("out of host memory");
    v.ld = c;
    return v;
}

/* X (r x c) copied into the leading block of an R x C matrix of zeros. */
static view_t zero_extend(const fmt_t *f, view_t X, int64_t r, int64_t c, int64_t R, int64_t C) {
    view_t Y = new_mat(f, R, C);
    for (int64_t i = 0; i < R; i++)
        for (int64_t j = 0; j < C; j++) {
            if (i < r && j < c) memcpy(at(f, Y, i, j), at(f, X, i, j), f->esz);
            else el_zero(f, at(f, Y, i, j));
        }
    return Y;
}

/* Eq 3, Strassen: P1..P7 exactly as written, then
   C11 = ((P1 + P4) - P5) + P7, C12 = P3 + P5, C21 = P2 + P4,
   C22 = ((P1 + P3) - P2) + P6, left to right.  `depth` levels of recursion;
   the leaves use the block algorithm with block size n_min.  Every dimension
   must be even at every level. */
static void gemm_strassen(const fmt_t *f, int64_t m, int64_t l, int64_t n, view_t A, view_t B, view_t C,
                          int64_t n_min, int depth) {
    if (depth <= 0) {
        gemm_block(f, m, l, n, A, B, C, n_min, 0, m);
        return;
    }
    if ((m | l | n) & 1) die("Strassen needs even dimensions at every level (the caller zero-extends)");
    int64_t m2 = m / 2, l2 = l / 2, n2 = n / 2;
    view_t A11 = sub_view(f, A, 0, 0), A12 = sub_view(f, A, 0, l2);
    view_t A21 = sub_view(f, A, m2, 0), A22 = sub_view(f, A, m2, l2);
    view_t B11 = sub_view(f, B, 0, 0), B12 = sub_view(f, B, 0, n2);
    view_t B21 = sub_view(f, B, l2, 0), B22 = sub_view(f, B, l2, n2);
    view_t C11 = sub_view(f, C, 0, 0), C12 = sub_view(f, C, 0, n2);
    view_t C21 = sub_view(f, C, m2, 0), C22 = sub_view(f, C, m2, n2);
    view_t S = new_mat(f, m2, l2), T = new_mat(f, l2, n2);
    view_t P[8];
    for (int i = 1; i <= 7; i++) P[i] = new_mat(f, m2, n2);

    mat_addsub(f, m2, l2, S, A11, A22, 0);                 /* P1 = (A11 + A22)(B11 + B22) */
    mat_addsub(f, l2, n2, T, B11, B22, 0);
    gemm_strassen(f, m2, l2, n2, S, T, P[1], n_min, depth - 1);
    mat_addsub(f, m2, l2, S, A21, A22, 0);                 /* P2 = (A21 + A22) B11 */
    gemm_strassen(f, m2, l2, n2, S, B11, P[2], n_min, depth - 1);
    mat_addsub(f, l2, n2, T, B12, B22, 1);                 /* P3 = A11 (B12 - B22) */
    gemm_strassen(f, m2, l2, n2, A11, T, P[3], n_min, depth - 1);
    mat_addsub(f, l2, n2, T, B21, B11, 1);                 /* P4 = A22 (B21 - B11) */
    gemm_strassen(f, m2, l2, n2, A22, T, P[4], n_min, depth - 1);
    mat_addsub(f, m2, l2, S, A11, A12, 0);                 /* P5 = (A11 + A12) B22 */
    gemm_strassen(f, m2, l2, n2, S, B22, P[5], n_min, depth - 1);
    mat_addsub(f, m2, l2, S, A21, A11, 1);                 /* P6 = (A21 - A11)(B11 + B12) */
    mat_addsub(f, l2, n2, T, B11, B12, 0);
    gemm_strassen(f, m2, l2, n2, S, T, P[6], n_min, depth - 1);
    mat_addsub(f, m2, l2, S, A12, A22, 1);                 /* P7 = (A12 - A22)(B21 + B22) */
    mat_addsub(f, l2, n2, T, B21, B22, 0);
    gemm_strassen(f, m2, l2, n2, S, T, P[7], n_min, depth - 1);

    mat_addsub(f, m2, n2, C11, P[1], P[4], 0);             /* C11 = P1 + P4 - P5 + P7 */
    mat_addsub(f, m2, n2, C11, C11, P[5], 1);
    mat_addsub(f, m2, n2, C11, C11, P[7], 0);
    mat_addsub(f, m2, n2, C12, P[3], P[5], 0);             /* C12 = P3 + P5 */
    mat_addsub(f, m2, n2, C21, P[2], P[4], 0);             /* C21 = P2 + P4 */
    mat_addsub(f, m2, n2, C22, P[1], P[3], 0);             /* C22 = P1 + P3 - P2 + P6 */
    mat_addsub(f, m2, n2, C22, C22, P[2], 1);
    mat_addsub(f, m2, n2, C22, C22, P[6], 0);

    free(S.p); free(T.p);
    for (int i = 1; i <= 7; i++) free(P[i].p);
}

/* ------------------------------------------------------------------------ */
/* Planes <-> AoS conversion and the exported GEMM entry points.            */
/* ------------------------------------------------------------------------ */

static int fmt_init(fmt_t *f, int kind, int prec_bits) {
    f->kind = kind;
    f->w = 0;
    if (kind == F_DD) f->esz = sizeof(dd_t);
    else if (kind == F_QD) f->esz = sizeof(qd_t);
    else {
        if (prec_bits <= 0 || prec_bits % 32 || prec_bits / 32 > MP_WMAX) return -1;
        f->w = prec_bits / 32;
        f->esz = sizeof(uint32_t) * (size_t)(2 + f->w);
    }
    return 0;
}

static int fmt_planes(const fmt_t *f) { return f->kind == F_DD ? 2 : f->kind == F_QD ? 4 : 2 + f->w; }

/* planes (rows x cols, `np` planes, 8-byte words for DD/QD, 4-byte for MP) -> AoS */
static view_t to_aos(const fmt_t *f, const void *planes, int64_t rows, int64_t cols) {
    view_t v = new_mat(f, rows, cols);
    size_t N = (size_t)(rows * cols);
    int np = fmt_planes(f);
    for (size_t e = 0; e < N; e++) {
        char *dst = v.p + e * f->esz;
        for (int q = 0; q < np; q++) {
            if (f->kind == F_MP) ((uint32_t *)dst)[q] = ((const uint32_t *)planes)[q * N + e];
            else ((double *)dst)[q] = ((const double *)planes)[q * N + e];
        }
    }
    return v;
}

static void from_aos_rows(const fmt_t *f, view_t v, void *planes, int64_t rows, int64_t cols, int64_t r0, int64_t r1) {
    size_t N = (size_t)(rows * cols);
    int np = fmt_planes(f);
    for (int64_t i = r0; i < r1; i++)
        for (int64_t j = 0; j < cols; j++) {
            size_t e = (size_t)(i * cols + j);
            const char *src = v.p + e * f->esz;
            for (int q = 0; q < np; q++) {
                if (f->kind == F_MP) ((uint32_t *)planes)[q * N + e] = ((const uint32_t *)src)[q];
                else ((double *)planes)[q * N + e] = ((const double *)src)[q];
            }
        }
}

enum { ALGO_SIMPLE = 0, ALGO_BLOCK = 1, ALGO_STRASSEN = 2 };

/* Generic driver.  Rows [r0, r1) of C are computed (simple and block only;
   Strassen always computes all of C).  Returns 0, or -1 on bad arguments. */
static int gemm_any(int kind, int prec_bits, int algo, int64_t m, int64_t l, int64_t n, const void *A,
                    const void *B, void *C, int64_t n_min, int depth, int64_t r0, int64_t r1) {
    fmt_t f;
    if (fmt_init(&f, kind, prec_bits)) return -1;
    if (m < 0 || l < 0 || n < 0) return -1;
    if (r0 < 0) r0 = 0;
    if (r1 < 0 || r1 > m) r1 = m;
    if (algo == ALGO_STRASSEN) { r0 = 0; r1 = m; }
    if (m == 0 || n == 0 || r1 <= r0) return 0;
    if (n_min <= 0) n_min = 64;
    view_t a = to_aos(&f, A, m, l), b = to_aos(&f, B, l, n), c = new_mat(&f, m, n);
    if (algo == ALGO_SIMPLE) gemm_simple(&f, m, l, n, a, b, c, r0, r1);
    else if (algo == ALGO_BLOCK) gemm_block(&f, m, l, n, a, b, c, n_min, r0, r1);
    else {
        /* Dimensions that 2^depth does not divide: A and B are extended with
           zero rows and columns to the next multiples of 2^depth, Eq 3 runs
           on the extended matrices and C is their product's leading m x n
           block (the paper runs Strassen at odd n without saying how). */
        int64_t q = (int64_t)1 << (depth > 0 ? depth : 0);
        int64_t mq = (m + q - 1) / q * q, lq = (l + q - 1) / q * q, nq = (n + q - 1) / q * q;
        view_t ap = zero_extend(&f, a, m, l, mq, lq), bp = zero_extend(&f, b, l, n, lq, nq);
        view_t cp = new_mat(&f, mq, nq);
        gemm_strassen(&f, mq, lq, nq, ap, bp, cp, n_min, depth);
        for (int64_t i = 0; i < m; i++)
            memcpy(at(&f, c, i, 0), at(&f, cp, i, 0), (size_t)n * f.esz);
        free(ap.p); free(bp.p); free(cp.p);
    }
    from_aos_rows(&f, c, C, m, n, r0, r1);
    free(a.p); free(b.p); free(c.p);
    return 0;
}

OR_API int or_dd_gemm(int algo, int64_t m, int64_t l, int64_t n, const double *A, const double *B, double *C,
                      int64_t n_min, int depth, int64_t r0, int64_t r1) {
    return gemm_any(F_DD, 0, algo, m, l, n, A, B, C, n_min, depth, r0, r1);
}
OR_API int or_qd_gemm(int algo, int64_t m, int64_t l, int64_t n, const double *A, const double *B, double *C,
                      int64_t n_min, int depth, int64_t r0, int64_t r1) {
    return gemm_any(F_QD, 0, algo, m, l, n, A, B, C, n_min, depth, r0, r1);
}
OR_API int or_mp_gemm(int prec_bits, int algo, int64_t m, int64_t l, int64_t n, const uint32_t *A,
                      const uint32_t *B, uint32_t *C, int64_t n_min, int depth, int64_t r0, int64_t r1) {
    return gemm_any(F_MP, prec_bits, algo, m, l, n, A, B, C, n_min, depth, r0, r1);
}

/* ------------------------------------------------------------------------ */
/* Exact checker for sampled entries of a DD or QD product.                 */
/* For each sample (i, j): err = RN(|c_exact - c_test|) and                 */
/* absab = RN(sum_k |a_ik| |b_kj|), both from exact accumulation, where the */
/* matrices hold `terms` planes (2 = DD, 4 = QD) and a value is the exact   */
/* sum of its terms.                                                         */
/* ------------------------------------------------------------------------ */

OR_API int or_exact_check(int terms, int64_t m, int64_t l, int64_t n, const double *A, const double *B,
                          const double *Ct, int64_t count, const int64_t *ii, const int64_t *jj, double *err,
                          double *absab) {
    size_t NA = (size_t)(m * l), NB = (size_t)(l * n), NC = (size_t)(m * n);
    if (terms != 2 && terms != 4) return -1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(or_get_threads())
    for (int64_t s = 0; s < count; s++) {
        int64_t i = ii[s], j = jj[s];
        wfx_t W, Wa;
        wfx_zero(&W);
        wfx_zero(&Wa);
        for (int64_t k = 0; k < l; k++) {
            double a[4], b[4];
            for (int q = 0; q < terms; q++) {
                a[q] = A[q * NA + (size_t)(i * l + k)];
                b[q] = B[q * NB + (size_t)(k * n + j)];
            }
            /* sign of a value = sign of its leading term (terms non-overlapping) */
            double sa = a[0] < 0 ? -1.0 : 1.0, sb = b[0] < 0 ? -1.0 : 1.0;
            for (int p = 0; p < terms; p++)
                for (int q = 0; q < terms; q++) {
                    wfx_add_prod(&W, a[p], b[q]);
                    wfx_add_prod(&Wa, sa * a[p], sb * b[q]);
                }
        }
        for (int q = 0; q < terms; q++) wfx_add_double(&W, -Ct[q * NC + (size_t)(i * n + j)]);
        err[s] = fabs(wfx_round(&W));
        absab[s] = wfx_round(&Wa);
    }
    return 0;
}

/* Exact product entries rounded to `terms` greedy terms (for fixtures). */
OR_API int or_exact_entries(int terms, int64_t m, int64_t l, int64_t n, const double *A, const double *B,
                            int64_t count, const int64_t *ii, const int64_t *jj, double *out) {
    size_t NA = (size_t)(m * l), NB = (size_t)(l * n);
    (void)m;
#pragma omp parallel for schedule(dynamic, 1) num_threads(or_get_threads())
    for (int64_t s = 0; s < count; s++) {
        int64_t i = ii[s], j = jj[s];
        wfx_t W;
        wfx_zero(&W);
        for (int64_t k = 0; k < l; k++)
            for (int p = 0; p < terms; p++)
                for (int q = 0; q < terms; q++)
                    wfx_add_prod(&W, A[p * NA + (size_t)(i * l + k)], B[q * NB + (size_t)(k * n + j)]);
        wfx_round_terms(&W, out + s * terms, terms);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Split-precision DD GEMM (Ozaki-style), step by step.                     */
/*  1. e_i = max_k expo(hi(a_ik)), f_j = max_k expo(hi(b_kj)), expo(x) the   */
/*     frexp exponent (x = f 2^expo, 0.5 <= |f| < 1); 0 for an all-zero row. */
/*  2. a'_ik = a_ik 2^-e_i (exact, |a'| < 1); digits by truncation:         */
/*     x = a'; for s = 1..S: d_s = trunc(128 x), x = 128 x - d_s,           */
/*     so sum_s d_s 2^(-7s) is a' truncated toward zero to 7S bits and every */
/*     d_s lies in [-127, 127] (int8).                                       */
/*  3. For every slice pair (s, t) with s + t <= S + 1, the integer product  */
/*     D_s^A D_t^B (exact, int32 range for l <= 133000), summed exactly per  */
/*     level g = s + t into L_g (int64).                                     */
/*  4. c_ij = RN_DD( 2^(e_i + f_j) * sum_g L_g(i,j) 2^(-7g) ), RN_DD(x) =    */
/*     (RN(x), RN(x - RN(x))).                                               */
/* ------------------------------------------------------------------------ */

static int frexp_expo(double x) {
    int e;
    if (x == 0.0) return INT32_MIN;
    frexp(x, &e);
    return e;
}

/* rows: per-row max over the `cols` entries of the hi plane (stride 1);
   cols: per-column max over rows (stride cols). */
OR_API void or_ozaki_row_expo(int64_t rows, int64_t cols, const double *hi, int32_t *e) {
    for (int64_t i = 0; i < rows; i++) {
        int mx = INT32_MIN;
        for (int64_t k = 0; k < cols; k++) {
            int t = frexp_expo(hi[i * cols + k]);
            if (t > mx) mx = t;
        }
        e[i] = mx == INT32_MIN ? 0 : mx;
    }
}
OR_API void or_ozaki_col_expo(int64_t rows, int64_t cols, const double *hi, int32_t *f) {
    for (int64_t j = 0; j < cols; j++) {
        int mx = INT32_MIN;
        for (int64_t k = 0; k < rows; k++) {
            int t = frexp_expo(hi[k * cols + j]);
            if (t > mx) mx = t;
        }
        f[j] = mx == INT32_MIN ? 0 : mx;
    }
}

/* Truncation toward zero of the exact value hi + lo of a DD. */
static double dd_trunc(double hi, double lo) {
    double t = trunc(hi);
    if (t == hi) {
        /* hi is an integer: lo decides whether hi + lo crosses it */
        if (hi > 0 && lo < 0) t = hi - 1.0;
        else if (hi < 0 && lo > 0) t = hi + 1.0;
        else if (hi == 0) t = 0.0;   /* |lo| < 1 */
    }
    return t;
}

/* One element: S digits of x = (hi + lo) 2^-e.  All steps exact. */
static void ozaki_digits(double hi, double lo, int e, int S, int8_t *d, int64_t stride) {
    double xh = ldexp(hi, -e), xl = ldexp(lo, -e);
    for (int s = 0; s < S; s++) {
        double yh = ldexp(xh, 7), yl = ldexp(xl, 7);
        double t = dd_trunc(yh, yl);
        if (t > 127.0 || t < -127.0) die("ozaki digit out of range");
        d[(int64_t)s * stride] = (int8_t)t;
        /* (yh - t) is exact (same sign, |yh - t| < |yh|); re-normalise exactly */
        two_sum(yh - t, yl, &xh, &xl);
    }
}

/* Digits of A (row-scaled; D is S planes of rows x cols int8) or of B
   (column-scaled when by_col != 0). */
OR_API void or_ozaki_slice(int by_col, int64_t rows, int64_t cols, const double *X, const int32_t *expo, int S,
                           int8_t *D) {
    size_t N = (size_t)(rows * cols);
    for (int64_t i = 0; i < rows; i++)
        for (int64_t j = 0; j < cols; j++) {
            size_t e = (size_t)(i * cols + j);
            ozaki_digits(X[e], X[N + e], by_col ? expo[j] : expo[i], S, D + e, (int64_t)N);
        }
}

/* Level sums: L has (2S + 1) planes of m x n int64; plane g holds L_g for
   g = 2..S+1 (other planes zero). */
OR_API void or_ozaki_levels(int64_t m, int64_t l, int64_t n, int S, const int8_t *DA, const int8_t *DB, int64_t *L) {
    size_t NA = (size_t)(m * l), NB = (size_t)(l * n), NC = (size_t)(m * n);
    memset(L, 0, sizeof(int64_t) * NC * (size_t)(2 * S + 1));
    for (int s = 1; s <= S; s++)
        for (int t = 1; s + t <= S + 1; t++) {
            const int8_t *a = DA + (size_t)(s - 1) * NA, *b = DB + (size_t)(t - 1) * NB;
            int64_t *Lg = L + (size_t)(s + t) * NC;
            for (int64_t i = 0; i < m; i++)
                for (int64_t j = 0; j < n; j++) {
                    int64_t acc = 0;
                    for (int64_t k = 0; k < l; k++) acc += (int64_t)a[i * l + k] * (int64_t)b[k * n + j];
                    if (acc > INT32_MAX || acc < INT32_MIN) die("slice product beyond int32");
                    Lg[i * n + j] += acc;
                }
        }
}

OR_API void or_ozaki_recombine(int64_t m, int64_t n, int S, const int64_t *L, const int32_t *e, const int32_t *f,
                               double *C) {
    size_t NC = (size_t)(m * n);
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++) {
            wfx_t W;
            double r[2];
            wfx_zero(&W);
            for (int g = 2; g <= S + 1; g++) {
                int64_t v = L[(size_t)g * NC + (size_t)(i * n + j)];
                if (v > (1LL << 53) || v < -(1LL << 53)) die("level sum beyond 2^53");
                wfx_add_double(&W, ldexp((double)v, e[i] + f[j] - 7 * g));
            }
            wfx_round_terms(&W, r, 2);
            C[i * n + j] = r[0];
            C[NC + (size_t)(i * n + j)] = r[1];
        }
}

/* Balanced base-32 digits (the FP8 variant of step 2): with one bit of
   headroom, x = a 2^-(e+1) (|x| < 1/2) is truncated toward zero to 5S bits
   by S base-32 truncation steps (d_s = trunc(32 x), x = 32 x - d_s, all
   exact), then the digits of |x| are balanced from the least significant
   up: a digit >= 16 becomes digit - 32 and carries 1 into the next more
   significant digit; the most significant digit keeps its carry (it stays
   <= 16 because |x| < 1/2).  Every digit lies in [-16, 16] (exact in FP8
   e4m3) and sum_s d_s 32^(S-s) = trunc(x 2^(5S)). */
static void ozaki_digits_b32(double hi, double lo, int e, int S, int8_t *d, int64_t stride) {
    double xh = ldexp(hi, -(e + 1)), xl = ldexp(lo, -(e + 1));
    int mag[64];
    int neg = (xh < 0) || (xh == 0 && xl < 0);
    if (S < 1 || S > 64) die("slice count out of range");
    for (int s = 0; s < S; s++) {
        double yh = ldexp(xh, 5), yl = ldexp(xl, 5);
        double t = dd_trunc(yh, yl);
        mag[s] = (int)fabs(t);
        if (mag[s] > 31) die("base-32 digit out of range");
        two_sum(yh - t, yl, &xh, &xl);
    }
    for (int s = S - 1; s >= 1; s--) {
        if (mag[s] >= 16) {
            mag[s] -= 32;
            mag[s - 1] += 1;
        }
    }
    if (mag[0] > 16) die("balanced top digit out of range");
    for (int s = 0; s < S; s++) d[(int64_t)s * stride] = (int8_t)(neg ? -mag[s] : mag[s]);
}

OR_API void or_ozaki_slice_b32(int by_col, int64_t rows, int64_t cols, const double *X, const int32_t *expo, int S,
                               int8_t *D) {
    size_t N = (size_t)(rows * cols);
    for (int64_t i = 0; i < rows; i++)
        for (int64_t j = 0; j < cols; j++) {
            size_t e = (size_t)(i * cols + j);
            ozaki_digits_b32(X[e], X[N + e], by_col ? expo[j] : expo[i], S, D + e, (int64_t)N);
        }
}

/* Step 4 for digits of `bits` bits with `head` bits of headroom per side:
   c_ij = RN_DD(2^(e_i + f_j + 2 head) sum_g L_g 2^(-bits g)). */
OR_API void or_ozaki_recombine_bits(int64_t m, int64_t n, int S, int bits, int head, const int64_t *L,
                                    const int32_t *e, const int32_t *f, double *C) {
    size_t NC = (size_t)(m * n);
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++) {
            wfx_t W;
            double r[2];
            wfx_zero(&W);
            for (int g = 2; g <= S + 1; g++) {
                int64_t v = L[(size_t)g * NC + (size_t)(i * n + j)];
                if (v > (1LL << 53) || v < -(1LL << 53)) die("level sum beyond 2^53");
                wfx_add_double(&W, ldexp((double)v, e[i] + f[j] + 2 * head - bits * g));
            }
            wfx_round_terms(&W, r, 2);
            C[i * n + j] = r[0];
            C[NC + (size_t)(i * n + j)] = r[1];
        }
}

/* Balanced base-32 digits of a T-term expansion x = x_0 + ... + x_{T-1}
   (T = 2: DD, T = 4: QD), the same definition as ozaki_digits_b32 computed
   another way: the exact sum is formed in the wide fixed-point accumulator,
   its magnitude's bits e, e-1, ..., e+1-5S (the first 5S bits of
   |x| 2^-(e+1), i.e. trunc toward zero) are read as S 5-bit digits from the
   most significant down, balanced from the least significant up (a digit
   >= 16 becomes digit - 32 and carries one), and given x's sign. */
static void ozaki_digits_b32_terms(const double *x, int64_t xstride, int T, int e, int S, int8_t *d,
                                   int64_t stride) {
    wfx_t W;
    int mag[96];
    int neg;
    if (S < 1 || S > 96) die("slice count out of range");
    wfx_zero(&W);
    for (int t = 0; t < T; t++) wfx_add_double(&W, x[(int64_t)t * xstride]);
    neg = wfx_is_neg(&W);
    if (neg) wfx_negate(&W);
    const int top = WFX_FRAC + e + 1;                /* window index of 2^(e+1) */
    if (top - 5 * S < 0) die("digits below the exact accumulator's window");
    if (top < WFX_LIMBS * 32 - 1 && wfx_bits(&W, top, 32) != 0) die("value not below 2^(e+1)");
    for (int s = 0; s < S; s++) mag[s] = (int)wfx_bits(&W, top - 5 * (s + 1), 5);
    for (int s = S - 1; s >= 1; s--) {
        if (mag[s] >= 16) {
            mag[s] -= 32;
            mag[s - 1] += 1;
        }
    }
    if (mag[0] > 16) die("balanced top digit out of range");
    for (int s = 0; s < S; s++) d[(int64_t)s * stride] = (int8_t)(neg ? -mag[s] : mag[s]);
}

/* Digits of a T-plane matrix X (rows x cols per plane), row (A) or column
   (B) scaled, as S planes of rows x cols int8 (B not transposed). */
OR_API void or_ozaki_slice_b32_terms(int by_col, int T, int64_t rows, int64_t cols, const double *X,
                                     const int32_t *expo, int S, int8_t *D) {
    size_t N = (size_t)(rows * cols);
    for (int64_t i = 0; i < rows; i++)
        for (int64_t j = 0; j < cols; j++) {
            size_t e = (size_t)(i * cols + j);
            ozaki_digits_b32_terms(X + e, (int64_t)N, T, by_col ? expo[j] : expo[i], S, D + e, (int64_t)N);
        }
}

/* Step 4 rounded to T terms: c_ij = the greedy T-term rounding (x_0 =
   RN(x), x_1 = RN(x - x_0), ...) of x = 2^(e_i + f_j + 2 head) sum_g L_g
   2^(-bits g), summed exactly.  C has T planes. */
OR_API void or_ozaki_recombine_terms(int64_t m, int64_t n, int S, int bits, int head, int T, const int64_t *L,
                                     const int32_t *e, const int32_t *f, double *C) {
    size_t NC = (size_t)(m * n);
    if (T < 1 || T > 8) die("bad term count");
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++) {
            wfx_t W;
            double r[8];
            wfx_zero(&W);
            for (int g = 2; g <= S + 1; g++) {
                int64_t v = L[(size_t)g * NC + (size_t)(i * n + j)];
                if (v > (1LL << 53) || v < -(1LL << 53)) die("level sum beyond 2^53");
                wfx_add_double(&W, ldexp((double)v, e[i] + f[j] + 2 * head - bits * g));
            }
            wfx_round_terms(&W, r, T);
            for (int t = 0; t < T; t++) C[(size_t)t * NC + (size_t)(i * n + j)] = r[t];
        }
}

/* The FP8-digit pipeline for T-term expansions (T = 2: DD, T = 4: QD):
   exponents of the leading plane, balanced base-32 digits, level sums,
   exact recombination rounded to T terms. */
OR_API int or_ozaki_gemm_b32_terms(int T, int64_t m, int64_t l, int64_t n, const double *A, const double *B,
                                   double *C, int S) {
    int32_t *e = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int32_t *f = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int8_t *DA = (int8_t *)malloc((size_t)(m * l * S) + 1);
    int8_t *DB = (int8_t *)malloc((size_t)(l * n * S) + 1);
    int64_t *L = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m * n) * (size_t)(2 * S + 1) + 8);
    if (!e || !f || !DA || !DB || !L) die("out of host memory");
    or_ozaki_row_expo(m, l, A, e);
    or_ozaki_col_expo(l, n, B, f);
    or_ozaki_slice_b32_terms(0, T, m, l, A, e, S, DA);
    or_ozaki_slice_b32_terms(1, T, l, n, B, f, S, DB);
    or_ozaki_levels(m, l, n, S, DA, DB, L);
    or_ozaki_recombine_terms(m, n, S, 5, 1, T, L, e, f, C);
    free(e); free(f); free(DA); free(DB); free(L);
    return 0;
}

/* The FP8-digit pipeline (steps 1, 2 with balanced base-32 digits, 3, 4). */
OR_API int or_ozaki_gemm_b32(int64_t m, int64_t l, int64_t n, const double *A, const double *B, double *C, int S) {
    int32_t *e = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int32_t *f = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int8_t *DA = (int8_t *)malloc((size_t)(m * l * S) + 1);
    int8_t *DB = (int8_t *)malloc((size_t)(l * n * S) + 1);
    int64_t *L = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m * n) * (size_t)(2 * S + 1) + 8);
    if (!e || !f || !DA || !DB || !L) die("out of host memory");
    or_ozaki_row_expo(m, l, A, e);
    or_ozaki_col_expo(l, n, B, f);
    or_ozaki_slice_b32(0, m, l, A, e, S, DA);
    or_ozaki_slice_b32(1, l, n, B, f, S, DB);
    or_ozaki_levels(m, l, n, S, DA, DB, L);
    or_ozaki_recombine_bits(m, n, S, 5, 1, L, e, f, C);
    free(e); free(f); free(DA); free(DB); free(L);
    return 0;
}

/* The whole split-precision pipeline (steps 1-4) for small sizes. */
OR_API int or_ozaki_gemm(int64_t m, int64_t l, int64_t n, const double *A, const double *B, double *C, int S) {
    int32_t *e = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    int32_t *f = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int8_t *DA = (int8_t *)malloc((size_t)(m * l * S) + 1);
    int8_t *DB = (int8_t *)malloc((size_t)(l * n * S) + 1);
    int64_t *L = (int64_t *)malloc(sizeof(int64_t) * (size_t)(m * n) * (size_t)(2 * S + 1) + 8);
    if (!e || !f || !DA || !DB || !L) die("out of host memory");
    or_ozaki_row_expo(m, l, A, e);
    or_ozaki_col_expo(l, n, B, f);
    or_ozaki_slice(0, m, l, A, e, S, DA);
    or_ozaki_slice(1, l, n, B, f, S, DB);
    or_ozaki_levels(m, l, n, S, DA, DB, L);
    or_ozaki_recombine(m, n, S, L, e, f, C);
    free(e); free(f); free(DA); free(DB); free(L);
    return 0;
}
