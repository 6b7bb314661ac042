// Device double-double (DD) and quad-double (QD) arithmetic for the GEMM
// kernels.  Every rounding is explicit (__dadd_rn / __dmul_rn / __fma_rn) so
// the compiler cannot contract or reassociate anything.
//
// The multiply-accumulate of the GEMM (Eq 1's c <- c + a_ik b_kj) uses a
// deferred-renormalisation accumulator instead of a full DD add per step:
//   DD:  state (s, t).  p = RN(ah bh) and its exact error e (TwoProd),
//        the two cross products accumulated into t with two FMAs, then
//        (s, r) = TwoSum(s, p) and t <- t + (e + r).  Every DD_RENORM steps
//        (s, t) = TwoSum(s, t).  5 FP64 operations per step: TwoProd (the
//        product and its error) and the error term of the exponent-ordered
//        TwoSum run on the integer pipe (the library DD add + multiply pair
//        costs 27).
//        Worst-case error after l steps: about (DD_RENORM + 3) l u^2 sum|a||b|
//        plus O(u^2) per product, inside the required 16 l u^2 |A||B|
//        (= 4 l 2^-104 |A||B|) for DD_RENORM = 8.
//   QD:  state (s0, s1, s2, s3), one level per order of magnitude u^k.
//        Products a_i b_j of order <= 2 are split exactly (TwoProd) and
//        every term of order <= 2 enters its level through TwoSum, its
//        rounding error going one level down; order-3 terms are added
//        plainly into s3 (their errors are order 4).  Every QD_RENORM steps
//        the levels are renormalised.  51.25 FP64 operations per step (the
//        six products of orders 0-2 through TwoProd, and the TwoSum errors of
//        orders 0 and 1 and of the renormalisation, on the integer pipe).  Worst case about
//        (10 QD_RENORM + 10) l u^4 sum|a||b|, inside 4 l 2^-208 = 64 l u^4.
#pragma once

#include <cuda_runtime.h>

namespace mpg {

#ifndef DD_RENORM
#define DD_RENORM 8
#endif
#ifndef QD_RENORM
#define QD_RENORM 4
#endif

// ---------------------------------------------------------------- EFTs

// The rounding error r = x + y - s of s = RN(x + y), exactly, for x whose
// exponent field is at least y's (Dekker's Fast2Sum condition), computed on
// the integer pipe instead of as y - (s - x) (2 FP64 operations).  With
// normal x, y, s and e(x) - e(y) <= 54: x, y and s are integer multiples of
// ulp(y), |r| <= ulp(s)/2 < 2^55 ulp(y), so r / ulp(y) is the 64-bit sum of
// the three scaled mantissas taken modulo 2^64; r is representable, so its
// double is assembled from that integer without rounding.  e(x) - e(y) > 54
// gives s = x and r = y; s below y's binade means the sum was exact (r = +0,
// as the FP64 formula gives).  Zero, subnormal, infinite or NaN operands and
// a subnormal r take the FP64 formula.  Bit-identical to y - (s - x)
// (checked on crafted and random pairs by mpgemm_selftest_two_sum).
__device__ __forceinline__ double fast_two_sum_err(double x, double y, double s) {
    const unsigned long long bx = (unsigned long long)__double_as_longlong(x);
    const unsigned long long by = (unsigned long long)__double_as_longlong(y);
    const unsigned long long bs = (unsigned long long)__double_as_longlong(s);
    const int Ex = (int)((bx >> 52) & 0x7ff), Ey = (int)((by >> 52) & 0x7ff), Es = (int)((bs >> 52) & 0x7ff);
    if (Ey == 0 || Ex == 0x7ff || Es == 0 || Es == 0x7ff) return __dsub_rn(y, __dsub_rn(s, x));
    const int dxy = Ex - Ey;
    if (dxy > 54) return y;
    if (Es < Ey) return 0.0;
    constexpr unsigned long long MM = (1ull << 52) - 1ull, H = 1ull << 52;
    unsigned long long X = ((bx & MM) | H) << dxy;          // x / ulp(y) mod 2^64
    unsigned long long Y = (by & MM) | H;                   // y / ulp(y)
    unsigned long long S = ((bs & MM) | H) << (Es - Ey);    // s / ulp(y) mod 2^64 (Es - Ey <= 55)
    if (bx >> 63) X = 0ull - X;
    if (by >> 63) Y = 0ull - Y;
    if (bs >> 63) S = 0ull - S;
    const long long ri = (long long)(X + Y - S);            // r / ulp(y), exact
    if (ri == 0) return 0.0;
    const unsigned long long m = ri < 0 ? 0ull - (unsigned long long)ri : (unsigned long long)ri;
    const int lz = __clzll((long long)m);
    const int F = Ey + 11 - lz;                             // exponent field of r
    if (F <= 0) return __dsub_rn(y, __dsub_rn(s, x));
    const unsigned long long mant = lz >= 11 ? m << (lz - 11) : m >> (11 - lz);
    return __longlong_as_double(
        (long long)((ri < 0 ? (1ull << 63) : 0ull) | ((unsigned long long)F << 52) | (mant & MM)));
}

// TwoProd on the integer pipe: p = RN(a b) and the exact error e = a b - p
// as the signed integer eu times 2^ge, from one 106-bit mantissa product
// P = Ma Mb (four 32 x 32-bit products of the 21- and 32-bit halves).  P is
// shifted left by sh = 0 or 1 into [2^105, 2^106); p's mantissa is
// q = RNE(P / 2^53) (guard bit 52, sticky bits 0-51, ties to even),
// 2^52 <= q <= 2^53 (q = 2^53 carries into the exponent field when the
// fields are packed as (E - 1) 2^52 + q), and e = P - q 2^53 = rem - up 2^53
// (rem = P mod 2^53, up = the rounding increment), |e| <= 2^52 units of
// 2^(Ea + Eb - 2150 - sh).  Returns false (p and e unspecified) for zero,
// subnormal, infinite or NaN operands and for exponent fields summing
// outside [1129, 3067] (products below 2^-917, or that may reach 2^1023):
// there the caller takes the FP64 operations.
__device__ __forceinline__ bool two_prod_i(double a, double b, double& p, long long& eu, int& ge) {
    const unsigned ah = (unsigned)__double2hiint(a), al = (unsigned)__double2loint(a);
    const unsigned bh = (unsigned)__double2hiint(b), bl = (unsigned)__double2loint(b);
    const int Ea = (int)((ah >> 20) & 0x7ffu), Eb = (int)((bh >> 20) & 0x7ffu);
    const bool ok = (unsigned)(Ea - 1) < 0x7feu && (unsigned)(Eb - 1) < 0x7feu && (unsigned)(Ea + Eb - 1129) <= 1938u;
    const unsigned a1 = (ah & 0xfffffu) | 0x100000u, b1 = (bh & 0xfffffu) | 0x100000u;
    const unsigned long long p00 = (unsigned long long)al * bl;
    const unsigned long long mid = (unsigned long long)al * b1 + (unsigned long long)a1 * bl;   // < 2^54
    const unsigned long long t = (p00 >> 32) + (mid & 0xffffffffull);
    const unsigned long long u = (unsigned long long)a1 * b1 + (mid >> 32) + (t >> 32);        // P / 2^64
    unsigned w0 = (unsigned)p00, w1 = (unsigned)t, w2 = (unsigned)u, w3 = (unsigned)(u >> 32);
    const int top = (int)(w3 >> 9);                          // bit 105 of P
    const int sh = 1 - top;
    w3 = __funnelshift_l(w2, w3, sh);
    w2 = __funnelshift_l(w1, w2, sh);
    w1 = __funnelshift_l(w0, w1, sh);
    w0 <<= sh;
    const unsigned qlo = __funnelshift_r(w1, w2, 21), qhi = __funnelshift_r(w2, w3, 21);
    const unsigned up = (w1 >> 20) & (((w1 & 0xfffffu) | w0) != 0u ? 1u : qlo) & 1u;
    const unsigned long long q = (((unsigned long long)qhi << 32) | qlo) + up;
    const int Ep = Ea + Eb - 1023 + top;                     // p's field before a rounding carry
    const unsigned sgn = (ah ^ bh) & 0x80000000u;
    p = __hiloint2double((int)(sgn | (((unsigned)(Ep - 1) << 20) + (unsigned)(q >> 32))), (int)(unsigned)q);
    const long long v = (long long)((((unsigned long long)(w1 & 0x1fffffu) << 32) | w0) - ((unsigned long long)up << 53));
    eu = sgn ? -v : v;
    ge = Ea + Eb - 2150 - sh;
    return ok;
}

// The double of the exact integer value eu 2^ge with |eu| <= 2^53 (no
// rounding needed); false for a subnormal result.
__device__ __forceinline__ bool exact_to_double(long long eu, int ge, double& e) {
    if (eu == 0) {
        e = 0.0;
        return true;
    }
    const unsigned long long m = eu < 0 ? 0ull - (unsigned long long)eu : (unsigned long long)eu;
    const int lz = __clzll((long long)m);                    // >= 10
    const int F = 63 - lz + ge + 1023;
    const unsigned long long mant = m << (lz - 11 >= 0 ? lz - 11 : 0) >> (lz - 11 >= 0 ? 0 : 11 - lz);
    e = __longlong_as_double((long long)((eu < 0 ? (1ull << 63) : 0ull) + ((unsigned long long)(F - 1) << 52) + mant));
    return F > 0;
}

// TwoProd: p = RN(a b) and e = a b - p exactly, both on the integer pipe
// (two_prod_i), the FP64 pair __dmul_rn / fma(a, b, -p) outside its range
// and for a subnormal e.  Bit-identical to the FP64 pair (checked against
// the host's IEEE product and the device FMA by mpgemm_selftest_two_prod).
__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
    long long eu;
    int ge;
    if (!(two_prod_i(a, b, p, eu, ge) && exact_to_double(eu, ge, e))) {
        p = __dmul_rn(a, b);
        e = __fma_rn(a, b, -p);
    }
}

// TwoSum: s = RN(a + b), e = a + b - s exactly, for any a, b.  Computed as
// Dekker's Fast2Sum after ordering the operands by their exponent fields,
// compared on the integer pipe, with the error term on the integer pipe as
// well: it returns exactly what Knuth's 6-operation TwoSum returns (both are
// error-free), with 1 FP64 operation instead of 6.  On GB300 the FP64 pipe
// (2 operations / clock / SM) is the bottleneck and the integer issue slots
// are otherwise idle.
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
    const int ea = __double2hiint(a) & 0x7ff00000, eb = __double2hiint(b) & 0x7ff00000;
    const bool sw = eb > ea;
    const double x = sw ? b : a, y = sw ? a : b;
    const double r = __dadd_rn(x, y);
    e = fast_two_sum_err(x, y, r);
    s = r;
}

// The FP64 form of the same: the reference for mpgemm_selftest_two_sum, and
// the QD MAC's order-2 TwoSums (where the integer pipe is already busy).
__device__ __forceinline__ void two_sum_fp64(double a, double b, double& s, double& e) {
    const int ea = __double2hiint(a) & 0x7ff00000, eb = __double2hiint(b) & 0x7ff00000;
    const bool sw = eb > ea;
    const double x = sw ? b : a, y = sw ? a : b;
    const double r = __dadd_rn(x, y);
    e = __dsub_rn(y, __dsub_rn(r, x));
    s = r;
}

// Dekker's Fast2Sum (exact when exponent(a) >= exponent(b)).
__device__ __forceinline__ void fast_two_sum(double a, double b, double& s, double& e) {
    double x = __dadd_rn(a, b);
    e = __dsub_rn(b, __dsub_rn(x, a));
    s = x;
}

// ---------------------------------------------------------------- DD

struct DDAcc {
    double s, t;
};

__device__ __forceinline__ void dd_zero(DDAcc& c) {
    c.s = 0.0;
    c.t = 0.0;
}

__device__ __forceinline__ void dd_mac(DDAcc& c, double ah, double al, double bh, double bl) {
    double p, e;
    two_prod(ah, bh, p, e);             // p = RN(ah bh) and its exact error, on the integer pipe
    double t = __fma_rn(ah, bl, c.t);   // cross products straight into the low part
    t = __fma_rn(al, bh, t);
    double s, r;
    two_sum(c.s, p, s, r);
    c.s = s;
    c.t = __dadd_rn(t, __dadd_rn(e, r));
}

// The DD MAC with every error term from FP64 operations (the reference of
// mpgemm_selftest_dd_mac).
__device__ __forceinline__ void dd_mac_fp64(DDAcc& c, double ah, double al, double bh, double bl) {
    const double p = __dmul_rn(ah, bh);
    const double e = __fma_rn(ah, bh, -p);
    double t = __fma_rn(ah, bl, c.t);
    t = __fma_rn(al, bh, t);
    double s, r;
    two_sum_fp64(c.s, p, s, r);
    c.s = s;
    c.t = __dadd_rn(t, __dadd_rn(e, r));
}

__device__ __forceinline__ void dd_renorm(DDAcc& c) {
    double s, t;
    two_sum(c.s, c.t, s, t);
    c.s = s;
    c.t = t;
}

// Accurate DD + DD (Joldes-Muller-Popescu 2017 "AccurateDWPlusDW", bound 3u^2),
// the rounding of each of the Strassen passes' sums and differences.  The
// passes compute it as dd_add_int (below: 8 FP64 operations) and use this
// form only for the operands that dd_add_int flags; here the TwoSums' FP64
// fallbacks, which the compiler predicates rather than branches around,
// bring the count to 12-18 FP64 instructions per addition (ncu), not 10.
__device__ __forceinline__ void dd_add(double xh, double xl, double yh, double yl, double& zh, double& zl) {
    double sh, sl, th, tl, vh, vl;
    two_sum(xh, yh, sh, sl);
    two_sum(xl, yl, th, tl);
    double c = __dadd_rn(sl, th);
    fast_two_sum(sh, c, vh, vl);
    double w = __dadd_rn(tl, vl);
    fast_two_sum(vh, w, zh, zl);
}

// ---------------------------------------------------------------- DD add, error terms on the integer pipe

__device__ __forceinline__ bool is_zero_bits(unsigned hi, unsigned lo) { return ((hi << 1) | lo) == 0u; }

// The rounding error r = x + y - s of s = RN(x + y) for x whose exponent
// field is at least y's, with no FP64 operation: the integer rule of
// fast_two_sum_err, and zeros handled exactly as the FP64 formula
// y - (s - x) treats them (y = +-0 gives r = y; s = +-0 with y != 0, i.e.
// x = -y, gives +0).  Where that formula would be needed instead (x or s
// infinite or NaN, y subnormal, r subnormal) `rare` is set and the value
// returned is unspecified: the caller recomputes with FP64 formulas.
// Zero tests use the 32-bit halves (a test on the 64-bit pattern can
// become an FP64 compare).
__device__ __forceinline__ double sum_err_int(double x, double y, double s, bool& rare) {
    const unsigned xh = (unsigned)__double2hiint(x), yh = (unsigned)__double2hiint(y);
    const unsigned sh = (unsigned)__double2hiint(s);
    const int Ex = (int)((xh >> 20) & 0x7ffu), Ey = (int)((yh >> 20) & 0x7ffu), Es = (int)((sh >> 20) & 0x7ffu);
    if (Ex == 0x7ff || Es == 0x7ff) {
        rare = true;
        return 0.0;
    }
    if (Ey == 0) {
        if (is_zero_bits(yh, (unsigned)__double2loint(y))) return y;
        rare = true;                                         // subnormal y
        return 0.0;
    }
    const int dxy = Ex - Ey;
    if (dxy > 54) return y;
    if (Es < Ey) return 0.0;                                 // exact sum (s = +-0 included)
    constexpr unsigned long long MM = (1ull << 52) - 1ull, H = 1ull << 52;
    const unsigned long long bx = (unsigned long long)__double_as_longlong(x);
    const unsigned long long by = (unsigned long long)__double_as_longlong(y);
    const unsigned long long bs = (unsigned long long)__double_as_longlong(s);
    unsigned long long X = ((bx & MM) | H) << dxy;          // x / ulp(y) mod 2^64
    unsigned long long Y = (by & MM) | H;                   // y / ulp(y)
    unsigned long long S = ((bs & MM) | H) << (Es - Ey);    // s / ulp(y) mod 2^64
    if (xh >> 31) X = 0ull - X;
    if (yh >> 31) Y = 0ull - Y;
    if (sh >> 31) S = 0ull - S;
    const long long ri = (long long)(X + Y - S);            // r / ulp(y), exact
    if (ri == 0) return 0.0;
    const unsigned long long m = ri < 0 ? 0ull - (unsigned long long)ri : (unsigned long long)ri;
    const int lz = __clzll((long long)m);
    const int F = Ey + 11 - lz;                             // exponent field of r
    if (F <= 0) {
        rare = true;                                         // subnormal r
        return 0.0;
    }
    const unsigned long long mant = lz >= 11 ? m << (lz - 11) : m >> (11 - lz);
    return __longlong_as_double(
        (long long)((ri < 0 ? (1ull << 63) : 0ull) | ((unsigned long long)F << 52) | (mant & MM)));
}

// TwoSum (operands ordered by exponent field, then Fast2Sum) with the error
// from sum_err_int: one FP64 operation; where `rare` stays false, s and e
// are those of two_sum bit for bit.
__device__ __forceinline__ void two_sum_int(double a, double b, double& s, double& e, bool& rare) {
    const int ea = __double2hiint(a) & 0x7ff00000, eb = __double2hiint(b) & 0x7ff00000;
    const bool sw = eb > ea;
    const double x = sw ? b : a, y = sw ? a : b;
    s = __dadd_rn(x, y);
    e = sum_err_int(x, y, s, rare);
}

// Dekker's Fast2Sum in the given operand order, error from sum_err_int: one
// FP64 operation.  Where e(a) >= e(b) the FP64 form b - (s - a) is exact and
// equals it; for a = +-0 (and finite b) that form gives +0; any other
// a with a smaller exponent field than b's (where the FP64 form need not be
// exact), or an infinite or NaN b, sets `rare`.  Where `rare` stays false,
// s and e are those of fast_two_sum bit for bit.
__device__ __forceinline__ void fast_two_sum_int(double a, double b, double& s, double& e, bool& rare) {
    const unsigned ah = (unsigned)__double2hiint(a), bh = (unsigned)__double2hiint(b);
    const int Ea = (int)((ah >> 20) & 0x7ffu), Eb = (int)((bh >> 20) & 0x7ffu);
    s = __dadd_rn(a, b);
    if (Ea >= Eb) {
        e = sum_err_int(a, b, s, rare);
    } else {
        e = 0.0;
        if (Eb == 0x7ff || !is_zero_bits(ah, (unsigned)__double2loint(a))) rare = true;
    }
}

// The accurate DD + DD of dd_add with three of its four error terms on the
// integer pipe (the two TwoSums' and the last Fast2Sum's): 8 FP64
// operations instead of 10.  The first Fast2Sum keeps dd_add's FP64 formula
// (the same bits by construction, whatever the operands' exponent order),
// which balances the FP64 and integer pipes of the Strassen passes (all
// four on the integer pipe: 6 FP64 operations, integer-issue bound).  Bit
// for bit dd_add's result wherever `rare` stays false (checked by
// mpgemm_selftest_dd_add); the caller recomputes with dd_add where it is set
// (infinite, NaN or subnormal values, and a last Fast2Sum whose operands
// are out of exponent order).
__device__ __forceinline__ void dd_add_int(double xh, double xl, double yh, double yl, double& zh, double& zl,
                                           bool& rare) {
    double sh, sl, th, tl, vh, vl;
    two_sum_int(xh, yh, sh, sl, rare);
    two_sum_int(xl, yl, th, tl, rare);
    const double c = __dadd_rn(sl, th);
    fast_two_sum(sh, c, vh, vl);
    const double w = __dadd_rn(tl, vl);
    fast_two_sum_int(vh, w, zh, zl, rare);
}

// -x by its sign bit (no FP64 operation).
__device__ __forceinline__ double neg_bits(double x) {
    return __hiloint2double(__double2hiint(x) ^ (int)0x80000000, __double2loint(x));
}

// ---------------------------------------------------------------- QD

struct QDAcc {
    double s0, s1, s2, s3;
};

__device__ __forceinline__ void qd_zero(QDAcc& c) {
    c.s0 = c.s1 = c.s2 = c.s3 = 0.0;
}

// Renormalise four levels: two TwoSum sweeps (bottom-up, then top-down);
// exact, the value is unchanged.
__device__ __forceinline__ void qd_renorm(QDAcc& c) {
    double a, b;
    two_sum(c.s2, c.s3, a, b); c.s2 = a; c.s3 = b;
    two_sum(c.s1, c.s2, a, b); c.s1 = a; c.s2 = b;
    two_sum(c.s0, c.s1, a, b); c.s0 = a; c.s1 = b;
    two_sum(c.s1, c.s2, a, b); c.s1 = a; c.s2 = b;
    two_sum(c.s2, c.s3, a, b); c.s2 = a; c.s3 = b;
}

// Final form: two renormalising sweeps, then one more top-down pass so the
// four terms come out non-overlapping for the values a GEMM produces.
__device__ __forceinline__ void qd_finish(QDAcc& c) {
    qd_renorm(c);
    qd_renorm(c);
    double a, b;
    two_sum(c.s0, c.s1, a, b); c.s0 = a; c.s1 = b;
    two_sum(c.s1, c.s2, a, b); c.s1 = a; c.s2 = b;
    two_sum(c.s2, c.s3, a, b); c.s2 = a; c.s3 = b;
}

__device__ __forceinline__ void qd_mac(QDAcc& c, const double a[4], const double b[4]) {
    double p, e, s, r;
    // order 0
    double e00;
    two_prod(a[0], b[0], p, e00);
    two_sum(c.s0, p, s, r);
    c.s0 = s;
    // order 1: r, e00, a0 b1, a1 b0 (into s1; errors -> order 2 terms)
    double l2a, l2b, l2c, l2d;
    two_sum(c.s1, r, s, l2a);
    c.s1 = s;
    two_sum(c.s1, e00, s, l2b);
    c.s1 = s;
    double e01;
    two_prod(a[0], b[1], p, e01);
    two_sum(c.s1, p, s, l2c);
    c.s1 = s;
    double e10;
    two_prod(a[1], b[0], p, e10);
    two_sum(c.s1, p, s, l2d);
    c.s1 = s;
    // order 2: l2a..l2d, e01, e10, a0 b2, a1 b1, a2 b0 (into s2; errors -> s3).
    // These nine TwoSums keep the FP64 error term: with all fourteen on the
    // integer pipe the QD MAC becomes integer-bound (measured: QD 1024^3
    // Strassen 99.3 ms all integer, 106.0 all FP64, 95.7 this split).
    double t3 = 0.0;
    two_sum_fp64(c.s2, l2a, s, r); c.s2 = s; t3 = __dadd_rn(t3, r);
    two_sum_fp64(c.s2, l2b, s, r); c.s2 = s; t3 = __dadd_rn(t3, r);
    two_sum_fp64(c.s2, l2c, s, r); c.s2 = s; t3 = __dadd_rn(t3, r);
    two_sum_fp64(c.s2, l2d, s, r); c.s2 = s; t3 = __dadd_rn(t3, r);
    two_sum_fp64(c.s2, e01, s, r); c.s2 = s; t3 = __dadd_rn(t3, r);
    two_sum_fp64(c.s2, e10, s, r); c.s2 = s; t3 = __dadd_rn(t3, r);
    two_prod(a[0], b[2], p, e);
    two_sum_fp64(c.s2, p, s, r); c.s2 = s; t3 = __dadd_rn(t3, __dadd_rn(r, e));
    two_prod(a[1], b[1], p, e);
    two_sum_fp64(c.s2, p, s, r); c.s2 = s; t3 = __dadd_rn(t3, __dadd_rn(r, e));
    two_prod(a[2], b[0], p, e);
    two_sum_fp64(c.s2, p, s, r); c.s2 = s; t3 = __dadd_rn(t3, __dadd_rn(r, e));
    // order 3: a0 b3 + a1 b2 + a2 b1 + a3 b0, plainly
    double q = __dmul_rn(a[3], b[0]);
    q = __fma_rn(a[2], b[1], q);
    q = __fma_rn(a[1], b[2], q);
    q = __fma_rn(a[0], b[3], q);
    c.s3 = __dadd_rn(c.s3, __dadd_rn(t3, q));
}

// z = x + y for QD (Strassen add/sub kernels).  Same level scheme as the MAC:
// levels 0-2 through TwoSum, level 3 plainly, then renormalised.
__device__ __forceinline__ void qd_add(const double x[4], const double y[4], double z[4]) {
    QDAcc c;
    double e0, t1, e1, t2, e2, f1, f2, g2;
    two_sum(x[0], y[0], c.s0, e0);
    two_sum(x[1], y[1], t1, e1);
    two_sum(x[2], y[2], t2, e2);
    double t3 = __dadd_rn(x[3], y[3]);
    two_sum(t1, e0, c.s1, f1);
    two_sum(t2, e1, c.s2, f2);
    double s2;
    two_sum(c.s2, f1, s2, g2);
    c.s2 = s2;
    c.s3 = __dadd_rn(__dadd_rn(t3, e2), __dadd_rn(f2, g2));
    qd_finish(c);
    z[0] = c.s0; z[1] = c.s1; z[2] = c.s2; z[3] = c.s3;
}

}  // namespace mpg
