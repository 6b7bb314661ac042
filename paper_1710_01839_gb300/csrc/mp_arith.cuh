// Device p-bit multi-limb binary floating point, p = 32 W, round to nearest
// with ties to even after every operation (the fixed-precision stand-in for
// MPFR, Section 4.2 of the paper).  One thread owns one value.  Up to 1024
// bits every loop is unrolled over compile-time limb indices so the limbs
// live in registers, and every data-dependent shift is a barrel shifter of
// selects (no dynamic register indexing); 2048-bit values keep their limbs
// in local memory, loop, and shift by direct limb indexing.
//
// Value: (-1)^sign * M * 2^(e - p), M in [2^(p-1), 2^p) (limb 0 least
// significant); zero has flag bit1 and M = 0, e = 0.  Exponents are carried
// in 64 bits during an operation and flagged when they leave int32.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mpg {

// Loops over limbs unroll completely while the value fits in registers (up
// to 32 limbs, 1024 bits); wider values (2048 bits) keep their limbs in
// local memory and loop.
#define MP_UNROLL _Pragma("unroll (W > 32 ? 1 : 128)")
#define MP_UNROLL_N _Pragma("unroll (N > 40 ? 1 : 128)")

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
// into sticky.  Register-resident values (N <= 40): limb moves by powers of
// two (selects, no dynamic register indexing), then a funnel shift.  Wider
// values live in local memory and move limbs by direct indexing.
template <int N>
__device__ __forceinline__ void shr_sticky(uint32_t (&v)[N], int d, uint32_t& sticky) {
    int q = d >> 5;
    if constexpr (N > 40) {
        if (q >= N) {
            for (int i = 0; i < N; i++) {
                sticky |= v[i];
                v[i] = 0u;
            }
        } else if (q > 0) {
            for (int i = 0; i < q; i++) sticky |= v[i];
            for (int i = 0; i < N; i++) v[i] = i + q < N ? v[i + q] : 0u;
        }
    } else {
#pragma unroll
        for (int st = 1; st < N; st <<= 1) {
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
        if (q >= N) {   // everything shifted out
            uint32_t all = 0;
#pragma unroll
            for (int i = 0; i < N; i++) all |= v[i];
            sticky |= all;
#pragma unroll
            for (int i = 0; i < N; i++) v[i] = 0u;
        }
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
    if constexpr (N > 40) {
        if (q > 0)
            for (int i = N - 1; i >= 0; i--) v[i] = i - q >= 0 ? v[i - q] : 0u;
    } else {
#pragma unroll
        for (int st = 1; st < N; st <<= 1) {
            bool on = (q & st) != 0;
#pragma unroll
            for (int i = N - 1; i >= 0; i--) {
                uint32_t nv = (i - st >= 0) ? v[i - st] : 0u;
                v[i] = on ? nv : v[i];
            }
        }
    }
    int r = s & 31;
    MP_UNROLL_N
    for (int i = N - 1; i > 0; i--) v[i] = __funnelshift_l(v[i - 1], v[i], r);
    v[0] = v[0] << r;
}

// Round-to-nearest-even increment of a W-limb mantissa; returns the carry out.
template <int W>
__device__ __forceinline__ bool round_up(uint32_t (&M)[W], bool inc) {
    uint32_t c = inc ? 1u : 0u;
MP_UNROLL
    for (int i = 0; i < W; i++) {
        uint32_t s = M[i] + c;
        c = (c && s == 0u) ? 1u : 0u;
        M[i] = s;
    }
    return c != 0u;
}

// r = RN_p(x * y).
template <int W>
__device__ __forceinline__ void mp_mul(const MPV<W>& x, const MPV<W>& y, MPV<W>& r, unsigned& status) {
    unsigned sign = (x.f ^ y.f) & 1u;
    if ((x.f | y.f) & 2u) {
        mp_set_zero(r, sign);
        return;
    }
    uint32_t P[2 * W];
MP_UNROLL
    for (int i = 0; i < 2 * W; i++) P[i] = 0u;
MP_UNROLL
    for (int i = 0; i < W; i++) {
        uint32_t carry = 0u;
MP_UNROLL
        for (int j = 0; j < W; j++) {
            uint64_t t = (uint64_t)x.m[i] * y.m[j] + P[i + j] + carry;
            P[i + j] = (uint32_t)t;
            carry = (uint32_t)(t >> 32);
        }
        P[i + W] = carry;
    }
    // P in [2^(2p-2), 2^(2p)): keep the top p bits after a shift of 0 or 1.
    int sh = (P[2 * W - 1] >> 31) ? 0 : 1;
    uint32_t M[W];
MP_UNROLL
    for (int i = 0; i < W; i++) M[i] = __funnelshift_l(P[W + i - 1], P[W + i], sh);
    uint32_t below = P[W - 1] << sh;          // bits under M, top bit = round bit
    uint32_t rb = below >> 31;
    uint32_t st = below << 1;
MP_UNROLL
    for (int i = 0; i < W - 1; i++) st |= P[i];
    bool inc = rb && (st != 0u || (M[0] & 1u));
    long long e = (long long)x.e + y.e - sh;
    if (round_up(M, inc)) {
        M[W - 1] = 0x80000000u;
        e += 1;
    }
    r.e = clamp_exp(e, status);
    r.f = sign;
MP_UNROLL
    for (int i = 0; i < W; i++) r.m[i] = M[i];
}

// r = RN_p(a + b).
template <int W>
__device__ __forceinline__ void mp_add(const MPV<W>& a, const MPV<W>& b, MPV<W>& r, unsigned& status) {
    constexpr int p = 32 * W;
    constexpr int N = W + 3;   // [guard, guard, M (W limbs), carry]
    if (a.f & 2u) {
        if (b.f & 2u) {
            mp_set_zero(r, a.f & b.f & 1u);
        } else {
            r = b;
        }
        return;
    }
    if (b.f & 2u) {
        r = a;
        return;
    }
    const bool sw = b.e > a.e;
    const int ex = sw ? b.e : a.e;
    const unsigned sx = (sw ? b.f : a.f) & 1u, sy = (sw ? a.f : b.f) & 1u;
    const long long d = (long long)ex - (sw ? a.e : b.e);
    if (d >= p + 2) {          // |y| below half an ulp of every neighbour of x
        r = sw ? b : a;
        return;
    }
    uint32_t X[N], Y[N];
    X[0] = X[1] = 0u;
    Y[0] = Y[1] = 0u;
MP_UNROLL
    for (int i = 0; i < W; i++) {
        X[i + 2] = sw ? b.m[i] : a.m[i];
        Y[i + 2] = sw ? a.m[i] : b.m[i];
    }
    X[N - 1] = 0u;
    Y[N - 1] = 0u;
    uint32_t sticky = 0u;
    if (d < 32) {
        // the common GEMM case: no limb moves, and the two guard limbs keep
        // every shifted-out bit (no sticky)
        const int r = (int)d;
MP_UNROLL
        for (int i = 0; i < N - 1; i++) Y[i] = __funnelshift_r(Y[i], Y[i + 1], r);
        Y[N - 1] >>= r;
    } else {
        shr_sticky<N>(Y, (int)d, sticky);
    }
    const bool stk = sticky != 0u;
    uint32_t S[N];
    unsigned sign = sx;
    if (sx == sy) {
        uint32_t c = 0u;
MP_UNROLL
        for (int i = 0; i < N; i++) {
            uint64_t t = (uint64_t)X[i] + Y[i] + c;
            S[i] = (uint32_t)t;
            c = (uint32_t)(t >> 32);
        }
    } else {
        // S = X - Y - stk; the dropped part of y then leaves a positive
        // remainder below S's last bit, kept as sticky.
        uint32_t br = stk ? 1u : 0u;
MP_UNROLL
        for (int i = 0; i < N; i++) {
            uint64_t t = (uint64_t)X[i] - Y[i] - br;
            S[i] = (uint32_t)t;
            br = (uint32_t)(t >> 63);
        }
        if (br) {   // only when d == 0 and My > Mx (exact): negate
            uint32_t c = 1u;
MP_UNROLL
            for (int i = 0; i < N; i++) {
                uint32_t v = ~S[i] + c;
                c = (c && v == 0u) ? 1u : 0u;
                S[i] = v;
            }
            sign = sy;
        }
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
        // leading bit to position p + 63 (top of limb N-2); a shift of 0 or 1
        // (no cancellation of the leading bits) is the common case
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
            s = p + 64 - L;
            shl<N>(S, s);
        }
        e = (long long)ex - s;
        sticky = 0u;
    }
    uint32_t M[W];
MP_UNROLL
    for (int i = 0; i < W; i++) M[i] = S[i + 2];
    uint32_t rb = S[1] >> 31;
    uint32_t st = (S[1] << 1) | S[0] | sticky | (stk ? 1u : 0u);
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
