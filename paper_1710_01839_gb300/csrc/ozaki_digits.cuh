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

// ---- T-term expansions (QD: T = 4) on NW 64-bit words.
//
// floor(|x| 2^sc) for a canonical expansion x = x_0 + ... + x_{T-1} (each
// term at most half an ulp of the one before, as the QD library keeps
// them): with y_t = sign(x) x_t, the terms that are integers after scaling
// add exactly; the first term with a fractional part adds its floor and
// ends the sum, because everything after it is smaller than half its ulp
// and so cannot move the floor.  The result is below 2^(64 NW).
template <int NW>
struct WideB32 {
    unsigned long long w[NW];
    bool neg;
};

// v += (neg ? -1 : 1) * M 2^q, 0 <= q < 64 NW.
template <int NW>
MPG_HD void wide_add_shifted(unsigned long long (&v)[NW], unsigned long long M, int q, bool neg) {
    const int k = q >> 6, b = q & 63;
    const unsigned long long lo = M << b, hi = b ? M >> (64 - b) : 0ull;
    unsigned long long c = neg ? 1ull : 0ull;   // two's complement of the addend when subtracting
    for (int i = 0; i < NW; i++) {
        // word i of M 2^q, by selects (no dynamically indexed array)
        const unsigned long long ti = i == k ? lo : (i == k + 1 ? hi : 0ull);
        const unsigned long long x = neg ? ~ti : ti;
        const unsigned long long s1 = v[i] + x;
        const unsigned long long c1 = s1 < v[i] ? 1ull : 0ull;
        const unsigned long long s2 = s1 + c;
        const unsigned long long c2 = s2 < s1 ? 1ull : 0ull;
        v[i] = s2;
        c = c1 | c2;
    }
}

template <int T, int NW>
MPG_HD void expansion_trunc_scaled(const double (&x)[T], int sc, WideB32<NW>& r) {
    bool sigma = false;   // sign of the expansion: that of its first nonzero term
    for (int t = T - 1; t >= 0; t--)
        if ((dbl_bits(x[t]) << 1) != 0ull) sigma = (dbl_bits(x[t]) >> 63) != 0ull;
    for (int i = 0; i < NW; i++) r.w[i] = 0ull;
    r.neg = sigma;
    for (int t = 0; t < T; t++) {
        unsigned long long M;
        int p;
        bool s;
        dbl_decode(x[t], M, p, s);
        if (M == 0ull) continue;
        const bool sub = s != sigma;
        const int q = p + sc;
        if (q >= 0) {
            if (q < 64 * NW) wide_add_shifted<NW>(r.w, M, q, sub);
            continue;
        }
        const unsigned long long ip = q > -64 ? M >> (-q) : 0ull;
        if (!frac_bits(M, q)) {
            if (ip) wide_add_shifted<NW>(r.w, ip, 0, sub);
            continue;
        }
        // the first term with a fraction: floor(y_t 2^sc), then stop
        if (!sub) {
            if (ip) wide_add_shifted<NW>(r.w, ip, 0, false);
        } else {
            wide_add_shifted<NW>(r.w, ip + 1ull, 0, true);
        }
        break;
    }
}

// C = 16 (1 + 32 + ... + 32^(S-2)) on NW words.
template <int NW>
MPG_HD void b32_bias_wide(int S, unsigned long long (&C)[NW]) {
    for (int i = 0; i < NW; i++) C[i] = 0ull;
    for (int k = 0; k < S - 1; k++) {
        const int b = 5 * k + 4;
        C[b >> 6] |= 1ull << (b & 63);
    }
}

template <int NW>
MPG_HD void b32_prepare_wide(WideB32<NW>& u, const unsigned long long (&C)[NW]) {
    unsigned long long c = 0ull;
    for (int i = 0; i < NW; i++) {
        const unsigned long long s1 = u.w[i] + C[i];
        const unsigned long long c1 = s1 < u.w[i] ? 1ull : 0ull;
        const unsigned long long s2 = s1 + c;
        const unsigned long long c2 = s2 < s1 ? 1ull : 0ull;
        u.w[i] = s2;
        c = c1 | c2;
    }
}

// 5-bit field K of U (K compile-time).
template <int K, int NW>
MPG_HD int b32_field_wide(const WideB32<NW>& u) {
    constexpr int b = 5 * K, k = b >> 6, r = b & 63;
    if constexpr (r <= 59) {
        return (int)((u.w[k] >> r) & 31ull);
    } else {
        const unsigned long long hi = k + 1 < NW ? u.w[k + 1] : 0ull;
        return (int)(((u.w[k] >> r) | (hi << (64 - r))) & 31ull);
    }
}

}  // namespace mpg
