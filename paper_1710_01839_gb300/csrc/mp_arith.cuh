// Device p-bit multi-limb binary floating point, p = 32 W, round to nearest
// with ties to even after every operation (the fixed-precision stand-in for
// MPFR, Section 4.2 of the paper).  One thread owns one value.  Every loop
// is unrolled over compile-time limb indices so the limbs live in
// registers, and every data-dependent shift is a barrel shifter of selects
// (no dynamic register indexing).  At 2048 bits the multiply's first
// operand is not held in registers but read limb by limb through an
// accessor (shared or global memory), which keeps a thread's live limbs
// (second operand, accumulator, high part of the product) within the
// register file.
//
// Value: (-1)^sign * M * 2^(e - p), M in [2^(p-1), 2^p) (limb 0 least
// significant); zero has flag bit1 and M = 0, e = 0.  Exponents are carried
// in 64 bits during an operation and flagged when they leave int32.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mpg {

// Loops over limbs unroll completely.
#define MP_UNROLL _Pragma("unroll")
#define MP_UNROLL_N _Pragma("unroll")

template <int W>
struct MPV {
    int e;
    unsigned f;   // bit0 sign, bit1 zero
    uint32_t m[W];
};

template <int W>
__device__ __forceinline__ void mp_set_zero(MPV<W>& r, unsigned sign) {
    r.e = 0;
    r.f = 2u | (sign & 1u);
MP_UNROLL
    for (int i = 0; i < W; i++) r.m[i] = 0u;
}

__device__ __forceinline__ int clamp_exp(long long e, unsigned& status) {
    if (e > 2147483647LL || e < -2147483647LL - 1) {
        status |= 1u;   // DEV_EXP_OVERFLOW
        return 0;
    }
    return (int)e;
}

// Shift the N-limb value v right by d >= 0 bits; OR of the dropped bits goes
// into sticky.  Limbs move by powers of two (selects, no dynamic register
// indexing), then a funnel shift.  QMAX: the caller guarantees that at most
// QMAX whole limbs move (d < 32 (QMAX + 1)), which drops the barrel stages
// above it.
template <int N, int QMAX = N>
__device__ __forceinline__ void shr_sticky(uint32_t (&v)[N], int d, uint32_t& sticky) {
    int q = d >> 5;
#pragma unroll
    for (int st = 1; st < N && st <= QMAX; st <<= 1) {
        bool on = (q & st) != 0;
        uint32_t drop = 0;
#pragma unroll
        for (int i = 0; i < st && i < N; i++) drop |= v[i];
        sticky |= on ? drop : 0u;
#pragma unroll
        for (int i = 0; i < N; i++) {
            uint32_t nv = (i + st < N) ? v[i + st] : 0u;
            v[i] = on ? nv : v[i];
        }
    }
    if (QMAX >= N && q >= N) {   // everything shifted out
        uint32_t all = 0;
#pragma unroll
        for (int i = 0; i < N; i++) all |= v[i];
        sticky |= all;
#pragma unroll
        for (int i = 0; i < N; i++) v[i] = 0u;
    }
    int r = d & 31;
    sticky |= r ? (v[0] << (32 - r)) : 0u;
    MP_UNROLL_N
    for (int i = 0; i < N - 1; i++) v[i] = __funnelshift_r(v[i], v[i + 1], r);
    v[N - 1] = v[N - 1] >> r;
}

// Shift the N-limb value v left by s >= 0 bits (zeros in, top bits dropped).
template <int N>
__device__ __forceinline__ void shl(uint32_t (&v)[N], int s) {
    int q = s >> 5;
#pragma unroll
    for (int st = 1; st < N; st <<= 1) {
        bool on = (q & st) != 0;
#pragma unroll
        for (int i = N - 1; i >= 0; i--) {
            uint32_t nv = (i - st >= 0) ? v[i - st] : 0u;
            v[i] = on ? nv : v[i];
        }
    }
    int r = s & 31;
    MP_UNROLL_N
    for (int i = N - 1; i > 0; i--) v[i] = __funnelshift_l(v[i - 1], v[i], r);
    v[0] = v[0] << r;
}

// S = X + Y over N limbs with one carry chain (add.cc / addc); the carry out
// of limb N - 1 is dropped (callers keep a zero top limb).
template <int N>
__device__ __forceinline__ void add_limbs(const uint32_t (&X)[N], const uint32_t (&Y)[N], uint32_t (&S)[N]) {
    asm volatile("add.cc.u32 %0, %1, %2;" : "=r"(S[0]) : "r"(X[0]), "r"(Y[0]));
#pragma unroll
    for (int i = 1; i < N - 1; i++) asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(S[i]) : "r"(X[i]), "r"(Y[i]));
    asm volatile("addc.u32 %0, %1, %2;" : "=r"(S[N - 1]) : "r"(X[N - 1]), "r"(Y[N - 1]));
}

// S = X - Y - b (b in {0, 1}) as X + ~Y + (1 - b) on one carry chain;
// returns 1 when the difference is negative (no carry out).
template <int N>
__device__ __forceinline__ uint32_t sub_limbs(const uint32_t (&X)[N], const uint32_t (&Y)[N], uint32_t b,
                                              uint32_t (&S)[N]) {
    uint32_t dummy, cout;
    asm volatile("add.cc.u32 %0, %1, 0xFFFFFFFF;" : "=r"(dummy) : "r"(1u - b));   // carry = 1 - b
#pragma unroll
    for (int i = 0; i < N; i++) asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(S[i]) : "r"(X[i]), "r"(~Y[i]));
    asm volatile("addc.u32 %0, 0, 0;" : "=r"(cout));
    return 1u - cout;
}

// Round-to-nearest-even increment of a W-limb mantissa; returns the carry out.
// The carry leaves limb 0 only when limb 0 was all ones (rare), so the walk
// over the upper limbs sits behind a branch.
template <int W>
__device__ __forceinline__ bool round_up(uint32_t (&M)[W], bool inc) {
    M[0] += inc ? 1u : 0u;
    if (inc && M[0] == 0u) {
        uint32_t c = 1u;
MP_UNROLL
        for (int i = 1; i < W; i++) {
            uint32_t s = M[i] + c;
            c = (c && s == 0u) ? 1u : 0u;
            M[i] = s;
        }
        return c != 0u;
    }
    return false;
}

// Exact product x y of two W-limb mantissas (limb 0 least significant),
// rounded to nearest even to W limbs: M, the normalising shift sh (0 or 1)
// and whether M must be incremented (before the carry out of round_up).
template <int W, bool INLINE_LOOPS>
__device__ __forceinline__ void mp_mul_exact_body(const uint32_t* xm, const uint32_t* ym, uint32_t* M, int& sh,
                                                  bool& inc) {
    uint32_t P[2 * W];
#pragma unroll(INLINE_LOOPS ? 128 : 1)
    for (int i = 0; i < 2 * W; i++) P[i] = 0u;
#pragma unroll(INLINE_LOOPS ? 128 : 1)
    for (int i = 0; i < W; i++) {
        uint32_t carry = 0u;
#pragma unroll(INLINE_LOOPS ? 128 : 1)
        for (int j = 0; j < W; j++) {
            uint64_t t = (uint64_t)xm[i] * ym[j] + P[i + j] + carry;
            P[i + j] = (uint32_t)t;
            carry = (uint32_t)(t >> 32);
        }
        P[i + W] = carry;
    }
    // P in [2^(2p-2), 2^(2p)): keep the top p bits after a shift of 0 or 1.
    sh = (P[2 * W - 1] >> 31) ? 0 : 1;
#pragma unroll(INLINE_LOOPS ? 128 : 1)
    for (int i = 0; i < W; i++) M[i] = __funnelshift_l(P[W + i - 1], P[W + i], sh);
    uint32_t below = P[W - 1] << sh;          // bits under M, top bit = round bit
    uint32_t rb = below >> 31;
    uint32_t st = below << 1;
#pragma unroll(INLINE_LOOPS ? 128 : 1)
    for (int i = 0; i < W - 1; i++) st |= P[i];
    inc = rb && (st != 0u || (M[0] & 1u));
}

// The same, out of line and on local memory, for the rare products whose
// high part leaves the rounding open (keeps the common path's registers).
template <int W>
__device__ __noinline__ void mp_mul_exact_slow(const uint32_t* xm, const uint32_t* ym, uint32_t* M, int* sh,
                                               int* inc) {
    int s;
    bool i;
    mp_mul_exact_body<W, false>(xm, ym, M, s, i);
    *sh = s;
    *inc = i ? 1 : 0;
}

// Limb accessors for the multiply's operands: limb(i), and quad(q) = limbs
// 4q .. 4q+3.
template <int W>
struct RegLimbs {   // limbs in registers
    static constexpr bool kQuads = false;
    const uint32_t (&m)[W];
    __device__ __forceinline__ uint32_t limb(int i) const { return m[i]; }
    __device__ __forceinline__ uint4 quad(int q) const {
        return make_uint4(m[4 * q], m[4 * q + 1], m[4 * q + 2], m[4 * q + 3]);
    }
};

struct SmemLimbs {  // limbs contiguous in shared memory, 16-byte aligned
    static constexpr bool kQuads = true;   // the multiply reads y four limbs per load
    const uint32_t* p;
    // volatile: every use loads again, so the operand never occupies registers
    __device__ __forceinline__ uint32_t limb(int i) const {
        uint32_t v;
        asm volatile("ld.volatile.shared.u32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(p + i)));
        return v;
    }
    __device__ __forceinline__ uint4 quad(int q) const {
        uint4 v;
        asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                     : "r"((unsigned)__cvta_generic_to_shared(p + 4 * q)));
        return v;
    }
};

// r = RN_p(x * y).  From W = 8 limbs up the high part of the product comes
// first: only the limb products of columns >= W - 2 (about half of the W^2),
// summed exactly.  The dropped products add less than W units of limb W - 1
// and limb W - 2 less than one more, so when limb W - 1's bits below M sit
// more than W + 1 units away from the half-ulp and from the next ulp, the
// rounding direction and M are those of the exact product (the test MPFR
// applies to its short products, Brent and Zimmermann, Modern Computer
// Arithmetic, Section 3.3.2); otherwise the full product is formed.
// The operands are given by exponent, flags and a limb accessor.
template <int W, class XA, class YA>
__device__ __forceinline__ void mp_mul_acc(int xe, unsigned xf, const XA& xa, int ye, unsigned yf, const YA& ya,
                                           MPV<W>& r, unsigned& status) {
    unsigned sign = (xf ^ yf) & 1u;
    if ((xf | yf) & 2u) {
        mp_set_zero(r, sign);
        return;
    }
    uint32_t M[W];
    int sh;
    bool inc;
    if constexpr (W >= 8) {
        static_assert(W % 4 == 0, "limb quads");
        uint32_t H[W + 2];   // limbs W-2 .. 2W-1 of the high part
MP_UNROLL
        for (int i = 0; i < W + 2; i++) H[i] = 0u;
MP_UNROLL
        for (int i = 0; i < W; i++) {
            const uint32_t xi = xa.limb(i);
            uint32_t carry = 0u;
MP_UNROLL
            for (int q = 0; q < W / 4; q++) {
                if (i + 4 * q + 3 >= W - 2) {   // constant after unrolling
                    uint32_t yv[4];
                    if constexpr (YA::kQuads) {
                        const uint4 y4 = ya.quad(q);
                        yv[0] = y4.x;
                        yv[1] = y4.y;
                        yv[2] = y4.z;
                        yv[3] = y4.w;
                    } else {
#pragma unroll
                        for (int u = 0; u < 4; u++) yv[u] = ya.limb(4 * q + u);
                    }
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const int j = 4 * q + u;
                        if (i + j >= W - 2) {
                            uint64_t t = (uint64_t)xi * yv[u] + H[i + j - (W - 2)] + carry;
                            H[i + j - (W - 2)] = (uint32_t)t;
                            carry = (uint32_t)(t >> 32);
                        }
                    }
                }
            }
            H[i + 2] = carry;
        }
        sh = (H[W + 1] >> 31) ? 0 : 1;
        const uint32_t ulp1 = sh ? 0x7FFFFFFFu : 0xFFFFFFFFu;   // one ulp of M, minus 1, in limb W-1
        const uint32_t half = sh ? 0x40000000u : 0x80000000u;
        const uint32_t u = H[1] & ulp1;                          // bits of limb W-1 below M
        if (u <= half - (W + 1) || (u > half && u <= ulp1 - W)) {
            inc = u > half;
MP_UNROLL
            for (int i = 0; i < W; i++) M[i] = __funnelshift_l(H[i + 1], H[i + 2], sh);
        } else {
            uint32_t xs[W], ys[W], Ms[W];
            int s2, i2;
MP_UNROLL
            for (int i = 0; i < W; i++) {
                xs[i] = xa.limb(i);
                ys[i] = ya.limb(i);
            }
            mp_mul_exact_slow<W>(xs, ys, Ms, &s2, &i2);
MP_UNROLL
            for (int i = 0; i < W; i++) M[i] = Ms[i];
            sh = s2;
            inc = i2 != 0;
        }
    } else {
        uint32_t xm[W], ym[W];
MP_UNROLL
        for (int i = 0; i < W; i++) {
            xm[i] = xa.limb(i);
            ym[i] = ya.limb(i);
        }
        mp_mul_exact_body<W, true>(xm, ym, M, sh, inc);
    }
    long long e = (long long)xe + ye - sh;
    if (round_up(M, inc)) {
        M[W - 1] = 0x80000000u;
        e += 1;
    }
    r.e = clamp_exp(e, status);
    r.f = sign;
MP_UNROLL
    for (int i = 0; i < W; i++) r.m[i] = M[i];
}

template <int W>
__device__ __forceinline__ void mp_mul(const MPV<W>& x, const MPV<W>& y, MPV<W>& r, unsigned& status) {
    mp_mul_acc<W>(x.e, x.f, RegLimbs<W>{x.m}, y.e, y.f, RegLimbs<W>{y.m}, r, status);
}

// r = RN_p(a + b).
//
// One code path for every exponent difference d and both signs, so that the
// threads of a warp (whose operands differ in d and sign at random in a
// GEMM) do not diverge: d is clamped to p + 2 (from there on |y| is below a
// quarter of x's ulp and the frame below rounds to x, which is RN(x + y) for
// every larger d as well), y is aligned by the barrel shifter, and the sum
// and the difference are one carry chain X + (Y xor mask) + carry-in.
// CLOSE: the operands are expected to be of similar magnitude (multi-limb
// images of DD / QD numbers); then when every active thread of the warp has
// d < 32 (a warp-wide decision, so no divergence) a plain funnel shift
// aligns y.  With exponents spread over a wide range the vote seldom
// succeeds and costs more than it saves, so the default leaves it out.
template <int W, bool CLOSE = false>
__device__ __forceinline__ void mp_add(const MPV<W>& a, const MPV<W>& b, MPV<W>& r, unsigned& status) {
    constexpr int p = 32 * W;
    constexpr int N = W + 2;   // [guard, M (W limbs), carry]
    if ((a.f | b.f) & 2u) {    // a zero operand (rare)
        if (a.f & 2u) {
            if (b.f & 2u) mp_set_zero(r, a.f & b.f & 1u);
            else r = b;
        } else {
            r = a;
        }
        return;
    }
    const bool sw = b.e > a.e;
    const int ex = sw ? b.e : a.e;
    const unsigned sx = (sw ? b.f : a.f) & 1u, sy = (sw ? a.f : b.f) & 1u;
    const long long dl = (long long)ex - (sw ? a.e : b.e);
    const int d = dl < p + 2 ? (int)dl : p + 2;
    uint32_t X[N], Y[N];
    X[0] = 0u;
    Y[0] = 0u;
MP_UNROLL
    for (int i = 0; i < W; i++) {
        X[i + 1] = sw ? b.m[i] : a.m[i];
        Y[i + 1] = sw ? a.m[i] : b.m[i];
    }
    X[N - 1] = 0u;
    Y[N - 1] = 0u;
    uint32_t sticky = 0u;
    if constexpr (CLOSE) {
        if (__all_sync(__activemask(), d < 32)) {
            // no limb moves, and the guard limb keeps every shifted-out bit
MP_UNROLL
            for (int i = 0; i < N - 1; i++) Y[i] = __funnelshift_r(Y[i], Y[i + 1], d);
            Y[N - 1] >>= d;
        } else {
            shr_sticky<N, W>(Y, d, sticky);   // d <= p + 2: at most W limbs move
        }
    } else {
        shr_sticky<N, W>(Y, d, sticky);   // d <= p + 2: at most W limbs move
    }
    const bool stk = sticky != 0u;
    // sum, or X - Y - stk (the dropped part of y then leaves a positive
    // remainder below S's last bit, kept as sticky) as X + ~Y + 1 - stk
    const bool sub = sx != sy;
    const uint32_t mask = sub ? 0xFFFFFFFFu : 0u;
    uint32_t S[N], dummy, cout;
    asm volatile("add.cc.u32 %0, %1, 0xFFFFFFFF;" : "=r"(dummy) : "r"((sub && !stk) ? 1u : 0u));
#pragma unroll
    for (int i = 0; i < N; i++) asm volatile("addc.cc.u32 %0, %1, %2;" : "=r"(S[i]) : "r"(X[i]), "r"(Y[i] ^ mask));
    asm volatile("addc.u32 %0, 0, 0;" : "=r"(cout));
    unsigned sign = sx;
    if (sub && !cout) {   // a borrow: only when d == 0 and My > Mx (exact): negate
        uint32_t c = 1u;
MP_UNROLL
        for (int i = 0; i < N; i++) {
            uint32_t v = ~S[i] + c;
            c = (c && v == 0u) ? 1u : 0u;
            S[i] = v;
        }
        sign = sy;
    }
    uint32_t nz = 0u;
MP_UNROLL
    for (int i = 0; i < N; i++) nz |= S[i];
    if (nz == 0u) {            // exact cancellation: +0
        mp_set_zero(r, 0u);
        return;
    }
    long long e;
    if (S[N - 1] != 0u) {      // carry out of M: one bit right
        sticky = (S[0] & 1u);
MP_UNROLL
        for (int i = 0; i < N - 1; i++) S[i] = __funnelshift_r(S[i], S[i + 1], 1);
        S[N - 1] >>= 1;
        e = (long long)ex + 1;
    } else {
        // leading bit to the top of limb N-2; a shift of 0 or 1 (no
        // cancellation of the leading bits) is the common case, and a larger
        // one happens only for d <= 1, where the sum is exact (the guard
        // limb then holds every bit, and with d >= 2 the shift is at most 1
        // with at least two guard bits below the round bit)
        int s;
        if (S[N - 2] >> 30) {
            s = (S[N - 2] >> 31) ? 0 : 1;
            if (s) {
MP_UNROLL
                for (int i = N - 1; i > 0; i--) S[i] = __funnelshift_l(S[i - 1], S[i], 1);
                S[0] <<= 1;
            }
        } else {
            int L = 0;
MP_UNROLL
            for (int i = 0; i < N - 1; i++)
                if (S[i]) L = 32 * i + 32 - __clz(S[i]);
            s = 32 * (N - 1) - L;
            shl<N>(S, s);
        }
        e = (long long)ex - s;
        sticky = 0u;
    }
    uint32_t M[W];
MP_UNROLL
    for (int i = 0; i < W; i++) M[i] = S[i + 1];
    uint32_t rb = S[0] >> 31;
    uint32_t st = (S[0] << 1) | sticky | (stk ? 1u : 0u);
    bool inc = rb && (st != 0u || (M[0] & 1u));
    if (round_up(M, inc)) {
        M[W - 1] = 0x80000000u;
        e += 1;
    }
    r.e = clamp_exp(e, status);
    r.f = sign;
MP_UNROLL
    for (int i = 0; i < W; i++) r.m[i] = M[i];
}

}  // namespace mpg
