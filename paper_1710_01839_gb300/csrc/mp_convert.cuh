// Conversions between doubles and p-bit multi-limb values (device side),
// used by the DD / QD GEMMs on the integer pipe (single and batched):
//   exact:  a finite double as a W-limb value (W >= 2 holds its 53 bits);
//   RN_53:  a W-limb value rounded to the nearest double, ties to even.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"
#include "mp_arith.cuh"

namespace mpg {

// x exactly as a W-limb value (W >= 2); non-finite x flags DEV_NONFINITE.
template <int W>
__device__ __forceinline__ void mp_from_double(double x, MPV<W>& r, unsigned& status) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 63);
    const int ef = (int)((b >> 52) & 0x7ff);
    uint64_t m = b & 0xFFFFFFFFFFFFFull;
    if (ef == 0x7ff) {
        status |= DEV_NONFINITE;
        mp_set_zero(r, sign);
        return;
    }
    if (ef == 0 && m == 0) {
        mp_set_zero(r, sign);
        return;
    }
    int k;   // x = m 2^k
    if (ef) {
        m |= 1ull << 52;
        k = ef - 1075;
    } else {
        k = -1074;
    }
    const int lz = __clzll((long long)m);
    m <<= lz;   // top bit at 63: x = m 2^(k - lz), and M = m 2^(p - 64)
#pragma unroll
    for (int i = 0; i < W - 2; i++) r.m[i] = 0u;
    r.m[W - 2] = (uint32_t)m;
    r.m[W - 1] = (uint32_t)(m >> 32);
    r.e = k - lz + 64;
    r.f = sign;
}

// RN_53 of a W-limb value (W >= 2).  The top 64 bits of M with the OR of
// the rest in bit 0 round to 53 bits exactly as M does (11 > 2 bits below
// the rounding position), and __ull2double_rn rounds to nearest even; the
// exponent field is then moved by e - 64.  Outside the normal range: ±0
// and DEV_EXP_OVERFLOW.
template <int W>
__device__ __forceinline__ double mp_to_double(const MPV<W>& v, unsigned& status) {
    if (v.f & 2u) return (v.f & 1u) ? -0.0 : 0.0;
    uint64_t top = ((uint64_t)v.m[W - 1] << 32) | v.m[W - 2];
    uint32_t st = 0u;
#pragma unroll
    for (int i = 0; i < W - 2; i++) st |= v.m[i];
    top |= st ? 1ull : 0ull;
    const double d = __ull2double_rn(top);   // in [2^63, 2^64]
    const uint64_t db = (uint64_t)__double_as_longlong(d);
    const long long field = (long long)((db >> 52) & 0x7ff) + (long long)v.e - 64;
    if (field < 1 || field > 2046) {
        status |= DEV_EXP_OVERFLOW;
        return (v.f & 1u) ? -0.0 : 0.0;
    }
    const uint64_t out = (db & ~(0x7ffull << 52)) | ((uint64_t)field << 52) | ((uint64_t)(v.f & 1u) << 63);
    return __longlong_as_double((long long)out);
}

// c = +0, then c = RN_p(c + x_t) for t = 0..T-1 (x_t = x[t * stride]).
template <int W, int T>
__device__ __forceinline__ void terms_to_mp(const double* x, int64_t stride, MPV<W>& c, unsigned& status) {
    mp_set_zero(c, 0u);
#pragma unroll
    for (int t = 0; t < T; t++) {
        MPV<W> v, s;
        mp_from_double<W>(x[t * stride], v, status);
        mp_add<W>(c, v, s, status);
        c = s;
    }
}

// The greedy expansion: x_t = RN_53(r), r = r - x_t (exact), t = 0..T-1,
// written to x[t * stride].
template <int W, int T>
__device__ __forceinline__ void mp_to_terms(MPV<W> r, double* x, int64_t stride, unsigned& status) {
#pragma unroll
    for (int t = 0; t < T; t++) {
        const double d = mp_to_double<W>(r, status);
        x[t * stride] = d;
        if (t + 1 < T) {
            MPV<W> v, s;
            mp_from_double<W>(-d, v, status);
            mp_add<W>(r, v, s, status);   // exact: r - RN_53(r) fits in p bits
            r = s;
        }
    }
}

}  // namespace mpg
