// Device double-double (DD) and quad-double (QD) arithmetic for the GEMM
// kernels.  Every rounding is explicit (__dadd_rn / __dmul_rn / __fma_rn) so
// the compiler cannot contract or reassociate anything.
//
// The multiply-accumulate of the GEMM (Eq 1's c <- c + a_ik b_kj) uses a
// deferred-renormalisation accumulator instead of a full DD add per step:
//   DD:  state (s, t).  p = RN(ah bh) and its exact error e from one FMA,
//        the two cross products accumulated into t with two more FMAs, then
//        (s, r) = TwoSum(s, p) and t <- t + (e + r).  Every DD_RENORM steps
//        (s, t) = TwoSum(s, t).  9 FP64 operations per step with the
//        exponent-ordered TwoSum below (the library DD add + multiply pair
//        costs 27).
//        Worst-case error after l steps: about (DD_RENORM + 3) l u^2 sum|a||b|
//        plus O(u^2) per product, inside the required 16 l u^2 |A||B|
//        (= 4 l 2^-104 |A||B|) for DD_RENORM = 8.
//   QD:  state (s0, s1, s2, s3), one level per order of magnitude u^k.
//        Products a_i b_j of order <= 2 are split exactly (TwoProd) and
//        every term of order <= 2 enters its level through TwoSum, its
//        rounding error going one level down; order-3 terms are added
//        plainly into s3 (their errors are order 4).  Every QD_RENORM steps
//        the levels are renormalised.  Worst case about
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

// TwoSum: s = RN(a + b), e = a + b - s exactly, for any a, b.  Computed as
// Dekker's Fast2Sum after ordering the operands by their exponent fields,
// compared on the integer pipe: it returns exactly what Knuth's 6-operation
// TwoSum returns (both are error-free), with 3 FP64 operations instead of 6.
// On GB300 the FP64 pipe (2 operations / clock / SM) is the bottleneck and
// the issue slots for the integer compare and selects are otherwise idle.
__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
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
    double p = __dmul_rn(ah, bh);
    double e = __fma_rn(ah, bh, -p);   // exact error of p
    double t = __fma_rn(ah, bl, c.t);   // cross products straight into the low part
    t = __fma_rn(al, bh, t);
    double s, r;
    two_sum(c.s, p, s, r);
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
// used by the Strassen add/sub kernels where each operation is rounded.
__device__ __forceinline__ void dd_add(double xh, double xl, double yh, double yl, double& zh, double& zl) {
    double sh, sl, th, tl, vh, vl;
    two_sum(xh, yh, sh, sl);
    two_sum(xl, yl, th, tl);
    double c = __dadd_rn(sl, th);
    fast_two_sum(sh, c, vh, vl);
    double w = __dadd_rn(tl, vl);
    fast_two_sum(vh, w, zh, zl);
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
    p = __dmul_rn(a[0], b[0]);
    double e00 = __fma_rn(a[0], b[0], -p);
    two_sum(c.s0, p, s, r);
    c.s0 = s;
    // order 1: r, e00, a0 b1, a1 b0 (into s1; errors -> order 2 terms)
    double l2a, l2b, l2c, l2d;
    two_sum(c.s1, r, s, l2a);
    c.s1 = s;
    two_sum(c.s1, e00, s, l2b);
    c.s1 = s;
    p = __dmul_rn(a[0], b[1]);
    double e01 = __fma_rn(a[0], b[1], -p);
    two_sum(c.s1, p, s, l2c);
    c.s1 = s;
    p = __dmul_rn(a[1], b[0]);
    double e10 = __fma_rn(a[1], b[0], -p);
    two_sum(c.s1, p, s, l2d);
    c.s1 = s;
    // order 2: l2a..l2d, e01, e10, a0 b2, a1 b1, a2 b0 (into s2; errors -> s3)
    double t3 = 0.0;
    two_sum(c.s2, l2a, s, r); c.s2 = s; t3 = __dadd_rn(t3, r);
    two_sum(c.s2, l2b, s, r); c.s2 = s; t3 = __dadd_rn(t3, r);
    two_sum(c.s2, l2c, s, r); c.s2 = s; t3 = __dadd_rn(t3, r);
    two_sum(c.s2, l2d, s, r); c.s2 = s; t3 = __dadd_rn(t3, r);
    two_sum(c.s2, e01, s, r); c.s2 = s; t3 = __dadd_rn(t3, r);
    two_sum(c.s2, e10, s, r); c.s2 = s; t3 = __dadd_rn(t3, r);
    p = __dmul_rn(a[0], b[2]);
    e = __fma_rn(a[0], b[2], -p);
    two_sum(c.s2, p, s, r); c.s2 = s; t3 = __dadd_rn(t3, __dadd_rn(r, e));
    p = __dmul_rn(a[1], b[1]);
    e = __fma_rn(a[1], b[1], -p);
    two_sum(c.s2, p, s, r); c.s2 = s; t3 = __dadd_rn(t3, __dadd_rn(r, e));
    p = __dmul_rn(a[2], b[0]);
    e = __fma_rn(a[2], b[0], -p);
    two_sum(c.s2, p, s, r); c.s2 = s; t3 = __dadd_rn(t3, __dadd_rn(r, e));
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
