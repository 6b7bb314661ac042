// Integer-only helpers of the FP8-digit split (host and device): the exact
// truncation of a scaled DD and its balanced base-32 digits.
#pragma once

#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define MPG_HD __host__ __device__ __forceinline__
#else
#define MPG_HD inline
#endif

namespace mpg {

MPG_HD unsigned long long dbl_bits(double x) {
#if defined(__CUDA_ARCH__)
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    std::memcpy(&b, &x, sizeof b);
    return b;
#endif
}

// ---- FP8 digits, integer arithmetic only (GB300 runs FP64 at a small
// fraction of its integer rate).
//
// T = trunc((hi + lo) 2^sc) exactly, sc = 5S - e - 1, for a DD with |lo| <=
// ulp(hi)/2: with H = hi 2^sc and L = lo 2^sc, T = trunc(H) when H has a
// fractional part (|L| is then too small to cross an integer), else T = H +
// trunc(L) when L has H's sign and H - ceil(|L|) sign(H) when it has the
// other one; T = trunc(L) when hi = 0.  |T| < 2^(5S-1) <= 2^119.

// x = (-1)^neg M 2^p for a finite double.
MPG_HD void dbl_decode(double x, unsigned long long& M, int& p, bool& neg) {
    const unsigned long long b = dbl_bits(x);
    neg = (b >> 63) != 0ull;
    int E = (int)((b >> 52) & 0x7ff);
    M = b & 0xFFFFFFFFFFFFFull;
    if (E) M |= 1ull << 52;
    else E = 1;
    p = E - 1075;
}

// trunc(M 2^q) as (h, l), 128 bits.
MPG_HD void shl_trunc128(unsigned long long M, int q, unsigned long long& h, unsigned long long& l) {
    if (q >= 128) {
        h = l = 0ull;
    } else if (q >= 64) {
        h = M << (q - 64);
        l = 0ull;
    } else if (q > 0) {
        h = M >> (64 - q);
        l = M << q;
    } else {
        h = 0ull;
        l = q > -64 ? M >> (-q) : 0ull;
    }
}

MPG_HD bool frac_bits(unsigned long long M, int q) {
    if (q >= 0 || M == 0ull) return false;
    return q <= -64 ? true : (M & ((1ull << (-q)) - 1ull)) != 0ull;
}

MPG_HD void dd_trunc_scaled(double hi, double lo, int sc, unsigned long long& th, unsigned long long& tl,
                            bool& neg) {
    unsigned long long Mh, Ml;
    int ph, pl;
    bool sh, sl;
    dbl_decode(hi, Mh, ph, sh);
    dbl_decode(lo, Ml, pl, sl);
    if (Mh == 0ull) {
        shl_trunc128(Ml, pl + sc, th, tl);
        neg = sl;
        return;
    }
    const int qh = ph + sc, ql = pl + sc;
    shl_trunc128(Mh, qh, th, tl);
    neg = sh;
    if (Ml == 0ull || frac_bits(Mh, qh)) return;
    unsigned long long ah, al;
    shl_trunc128(Ml, ql, ah, al);
    if (sl == sh) {
        const unsigned long long t = tl + al;
        th += ah + (t < tl ? 1ull : 0ull);
        tl = t;
    } else {
        if (frac_bits(Ml, ql)) {   // ceil(|L|)
            al += 1ull;
            ah += al == 0ull ? 1ull : 0ull;
        }
        const unsigned long long t = tl - al;
        th -= ah + (tl < al ? 1ull : 0ull);
        tl = t;
    }
}

// Balanced base-32 digits of |T| < 2^(5S-1): U = |T| + C with C = 16 (1 +
// 32 + ... + 32^(S-2)); digit k (k = 0 least significant) is field k of U
// minus 16 for k < S - 1, and field S - 1 of U itself (<= 16) for the top
// digit.  This is the digit set of the carry rule (a digit >= 16 becomes
// digit - 32 and carries one), read off without a carry loop.
struct B32 {
    unsigned long long h, l;
    bool neg;
};

MPG_HD B32 b32_prepare(double hi, double lo, int sc, unsigned long long Ch, unsigned long long Cl) {
    B32 r;
    dd_trunc_scaled(hi, lo, sc, r.h, r.l, r.neg);
    const unsigned long long t = r.l + Cl;
    r.h += Ch + (t < r.l ? 1ull : 0ull);
    r.l = t;
    return r;
}

template <int K>
MPG_HD int b32_field(const B32& u) {
    if constexpr (5 * K + 5 <= 64) return (int)((u.l >> (5 * K)) & 31ull);
    else if constexpr (5 * K >= 64) return (int)((u.h >> (5 * K - 64)) & 31ull);
    else return (int)(((u.l >> (5 * K)) | (u.h << (64 - 5 * K))) & 31ull);
}

// C = 16 (1 + 32 + ... + 32^(S-2)) as 128 bits.
MPG_HD void b32_bias(int S, unsigned long long& Ch, unsigned long long& Cl) {
    Ch = Cl = 0ull;
    for (int k = 0; k < S - 1; k++) {
        const int b = 5 * k + 4;   // bit of 16 * 32^k
        if (b < 64) Cl |= 1ull << b;
        else Ch |= 1ull << (b - 64);
    }
}

}  // namespace mpg
