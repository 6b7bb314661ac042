// Warp-cooperative p-bit multi-limb arithmetic (p = 32 W, W = 8 T): one
// value is held by a team of T consecutive lanes of a warp, lane t holding
// limbs 8t .. 8t + 7 (limb 0 least significant), the exponent and flags
// replicated in every lane of the team.  The operations and the value format
// are those of mp_arith.cuh (round to nearest even after every multiply and
// every add, the same special cases, the same bits); what differs is where
// the limbs live.  A lane holds 8 limbs instead of W, so a wide value costs a
// few dozen registers per lane, and whatever crosses limbs crosses lanes:
//
//  - the product is formed by operand scanning: every lane multiplies the
//    limbs of a, read by the whole team from shared memory, by its own 8
//    limbs of b into a 16-limb window; after each 8 limbs of a the window's
//    finished low half moves one lane down by warp shuffles and is added to
//    the neighbour's high half (the lowest lane's low halves are the
//    product's low limbs, kept only as round bit and sticky);
//  - carries between lanes are resolved at once by a look-ahead over two
//    warp ballots: with G the lanes whose own sum carried out (generate) and
//    P the lanes whose limbs are all ones (propagate), the carry into lane t
//    is bit t of (U + V) xor U xor V, U = G | P, V = G, with each team's top
//    lane cleared so that no carry crosses into the next team;
//  - a shift by d bits fetches each lane's window of source limbs from the
//    two or three lanes that hold them and selects within it.
//
// Every shuffle and ballot runs on all 32 lanes under warp-uniform control
// flow (teams whose operands are zero compute on and select at the end); the
// rare cases (a borrow that needs a negation, a cancellation of the leading
// bits, a carry past a lane's limbs) take branches decided for the whole warp.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mp_arith.cuh"

namespace mpg {

constexpr unsigned kWarpAll = 0xFFFFFFFFu;

// Bits of every team's top lane in a warp ballot.
template <int T>
__host__ __device__ constexpr unsigned team_top_lanes() {
    unsigned m = 0u;
    for (int k = T - 1; k < 32; k += T) m |= 1u << k;
    return m;
}

template <int T>
struct Team {
    static_assert(T == 2 || T == 4 || T == 8 || T == 16 || T == 32, "team size: a power of two up to 32");
    int t;      // lane within the team
    int base;   // warp lane of the team's lane 0
    __device__ __forceinline__ Team() {
        const int lane = (int)(threadIdx.x & 31u);
        t = lane & (T - 1);
        base = lane - t;
    }
    __device__ __forceinline__ unsigned bits() const {
        return (T == 32 ? kWarpAll : ((1u << (T & 31)) - 1u)) << base;
    }
    // the value of lane t + 1 (0 in the top lane)
    __device__ __forceinline__ uint32_t above(uint32_t v) const {
        const uint32_t x = __shfl_down_sync(kWarpAll, v, 1, T);
        return t == T - 1 ? 0u : x;
    }
    // the value of lane t - 1 (0 in lane 0)
    __device__ __forceinline__ uint32_t below(uint32_t v) const {
        const uint32_t x = __shfl_up_sync(kWarpAll, v, 1, T);
        return t == 0 ? 0u : x;
    }
    // the value of lane src of the team
    __device__ __forceinline__ uint32_t from(uint32_t v, int src) const { return __shfl_sync(kWarpAll, v, src, T); }
    // p on any lane of the team
    __device__ __forceinline__ bool any(bool p) const { return (__ballot_sync(kWarpAll, p) & bits()) != 0u; }
    // The carry into this lane from the lanes below it: g = this lane's own
    // sum carried out, p = its limbs are all ones (a carry in passes through);
    // g and p are never both set.  Lane 0 receives none.
    __device__ __forceinline__ uint32_t carry_in(bool g, bool p) const {
        const unsigned G = __ballot_sync(kWarpAll, g), P = __ballot_sync(kWarpAll, p);
        constexpr unsigned top = team_top_lanes<T>();
        const unsigned U = (G | P) & ~top, V = G & ~top;
        return (((U + V) ^ U ^ V) >> (base + t)) & 1u;
    }
};

__device__ __forceinline__ bool tm_all_ones(const uint32_t (&X)[8]) {
    return (X[0] & X[1] & X[2] & X[3] & X[4] & X[5] & X[6] & X[7]) == 0xFFFFFFFFu;
}

__device__ __forceinline__ bool tm_nonzero(const uint32_t (&X)[8]) {
    return (X[0] | X[1] | X[2] | X[3] | X[4] | X[5] | X[6] | X[7]) != 0u;
}

// X += c (c in {0, 1}) on one carry chain; returns the carry out.
__device__ __forceinline__ uint32_t tm_add_small(uint32_t (&X)[8], uint32_t c) {
    uint32_t co;
    asm("add.cc.u32 %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, 0;\n\t"
        "addc.cc.u32 %2, %2, 0;\n\t"
        "addc.cc.u32 %3, %3, 0;\n\t"
        "addc.cc.u32 %4, %4, 0;\n\t"
        "addc.cc.u32 %5, %5, 0;\n\t"
        "addc.cc.u32 %6, %6, 0;\n\t"
        "addc.cc.u32 %7, %7, 0;\n\t"
        "addc.u32 %8, 0, 0;"
        : "+r"(X[0]), "+r"(X[1]), "+r"(X[2]), "+r"(X[3]), "+r"(X[4]), "+r"(X[5]), "+r"(X[6]), "+r"(X[7]),
          "=r"(co)
        : "r"(c));
    return co;
}

// Add c (in {0, 1}) to the team value X at lane 0's limb 0 (in lanes other
// than 0, c must be 0) and carry through the lanes; returns the carry out of
// the team's top limb in every lane of the team.
template <int T>
__device__ __forceinline__ uint32_t tm_increment(uint32_t (&X)[8], uint32_t c, const Team<T>& tm) {
    uint32_t g = tm_add_small(X, c);
    uint32_t cout = 0u;
    if (__any_sync(kWarpAll, g != 0u)) {   // a carry left some lane (rare)
        const uint32_t k = tm.carry_in(g != 0u, tm_all_ones(X));
        const uint32_t g2 = tm_add_small(X, k);
        cout = tm.from(tm.t == T - 1 ? (g | g2) : 0u, T - 1);
    }
    return cout;
}

// w[u] = limb (8t + v + u) of the team value X, u = 0..9, for v the same in
// the whole team: limbs 0..W-1 from the lanes that hold them, limb -1 reads
// xm1 and every other limb outside [0, W) reads 0.
template <int T>
__device__ __forceinline__ void tm_window(const uint32_t (&X)[8], uint32_t xm1, int v, const Team<T>& tm,
                                          uint32_t (&w)[10]) {
    const int vh = v >> 3;   // floor(v / 8)
    const int vl = v & 7;
    uint32_t z[17];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const int a = tm.t + vh + j;
        const bool ok = a >= 0 && a < T;
        const int src = ok ? a : 0;
#pragma unroll
        for (int s = 0; s < (j < 2 ? 8 : 1); s++) {
            const uint32_t x = tm.from(X[s], src);
            z[8 * j + s] = ok ? x : ((a == -1 && s == 7) ? xm1 : 0u);
        }
    }
#pragma unroll
    for (int i = 0; i < 13; i++) z[i] = (vl & 4) ? z[i + 4] : z[i];
#pragma unroll
    for (int i = 0; i < 11; i++) z[i] = (vl & 2) ? z[i + 2] : z[i];
#pragma unroll
    for (int i = 0; i < 10; i++) z[i] = (vl & 1) ? z[i + 1] : z[i];
#pragma unroll
    for (int u = 0; u < 10; u++) w[u] = z[u];
}

// R[O .. O+8] += ai * b (R[O+8] is 0 on entry): one row of the operand
// scanning.  The 9-limb sum fits, so no carry is lost.  WIDE: 64-bit
// products with the running carry in a register (a wide multiply-add and
// integer adds per limb), else two carry chains of 32-bit multiply-adds
// (the low halves, then the high halves one limb up), which take fewer
// registers.
template <int O, bool WIDE>
__device__ __forceinline__ void tm_mad_row(uint32_t (&R)[16], uint32_t ai, const uint32_t (&b)[8]) {
    static_assert(O >= 0 && O + 8 < 16, "window");
    if constexpr (WIDE) {
        uint32_t carry = 0u;
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const uint64_t t = (uint64_t)ai * b[u] + R[O + u] + carry;
            R[O + u] = (uint32_t)t;
            carry = (uint32_t)(t >> 32);
        }
        R[O + 8] = carry;
    } else {
        asm("mad.lo.cc.u32 %0, %9, %10, %0;\n\t"
            "madc.lo.cc.u32 %1, %9, %11, %1;\n\t"
            "madc.lo.cc.u32 %2, %9, %12, %2;\n\t"
            "madc.lo.cc.u32 %3, %9, %13, %3;\n\t"
            "madc.lo.cc.u32 %4, %9, %14, %4;\n\t"
            "madc.lo.cc.u32 %5, %9, %15, %5;\n\t"
            "madc.lo.cc.u32 %6, %9, %16, %6;\n\t"
            "madc.lo.cc.u32 %7, %9, %17, %7;\n\t"
            "addc.u32 %8, 0, 0;\n\t"
            "mad.hi.cc.u32 %1, %9, %10, %1;\n\t"
            "madc.hi.cc.u32 %2, %9, %11, %2;\n\t"
            "madc.hi.cc.u32 %3, %9, %12, %3;\n\t"
            "madc.hi.cc.u32 %4, %9, %13, %4;\n\t"
            "madc.hi.cc.u32 %5, %9, %14, %5;\n\t"
            "madc.hi.cc.u32 %6, %9, %15, %6;\n\t"
            "madc.hi.cc.u32 %7, %9, %16, %7;\n\t"
            "madc.hi.u32 %8, %9, %17, %8;"
            : "+r"(R[O]), "+r"(R[O + 1]), "+r"(R[O + 2]), "+r"(R[O + 3]), "+r"(R[O + 4]), "+r"(R[O + 5]),
              "+r"(R[O + 6]), "+r"(R[O + 7]), "+r"(R[O + 8])
            : "r"(ai), "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
    }
}

// H += in + cx (cx in {0, 1}) on one carry chain; cx becomes the carry out.
__device__ __forceinline__ void tm_add_in(uint32_t* H, const uint32_t (&in)[8], uint32_t& cx) {
    asm("{\n\t.reg .u32 t;\n\t"
        "add.cc.u32 t, %8, 0xFFFFFFFF;\n\t"
        "addc.cc.u32 %0, %0, %9;\n\t"
        "addc.cc.u32 %1, %1, %10;\n\t"
        "addc.cc.u32 %2, %2, %11;\n\t"
        "addc.cc.u32 %3, %3, %12;\n\t"
        "addc.cc.u32 %4, %4, %13;\n\t"
        "addc.cc.u32 %5, %5, %14;\n\t"
        "addc.cc.u32 %6, %6, %15;\n\t"
        "addc.cc.u32 %7, %7, %16;\n\t"
        "addc.u32 %8, 0, 0;\n\t}"
        : "+r"(H[0]), "+r"(H[1]), "+r"(H[2]), "+r"(H[3]), "+r"(H[4]), "+r"(H[5]), "+r"(H[6]), "+r"(H[7]),
          "+r"(cx)
        : "r"(in[0]), "r"(in[1]), "r"(in[2]), "r"(in[3]), "r"(in[4]), "r"(in[5]), "r"(in[6]), "r"(in[7]));
}

__device__ __forceinline__ uint4 tm_lds4(const uint32_t* p) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
    return v;
}

// The exact product of the W-limb mantissas a (limbs at `al` in shared
// memory, 16-byte aligned, the same address in the whole team) and b (this
// lane's limbs bl): this lane's limbs of the high half, H = P[W + 8t ..
// W + 8t + 7], and, meaningful in lane 0, plast = P[W - 1] and stk = the OR
// of P[0 .. W - 2].
//
// Window: in block j (limbs 8j .. 8j + 7 of a) R[u] is column 8j + 8t + u
// of the product.  Row i = 8j + o adds a_i b into R[o .. o + 8]; the 9-limb
// sum fits (R[o .. o + 7] < 2^256 and R[o + 8] = 0 before it, a_i b <
// 2^288 - 2^256), so no carry is ever lost.  At the block's end R[0 .. 7]
// are final for this lane's part and belong to the columns of the lane
// below's R[8 .. 15]: they move down and are added there, the carry of that
// addition (cx) is added at the next block's end into R[8] of the next
// window, i.e. the same column.
template <int W>
__device__ __forceinline__ void tm_mul_full(const uint32_t* al, const uint32_t (&bl)[8], const Team<W / 8>& tm,
                                            uint32_t (&H)[8], uint32_t& plast, uint32_t& stk) {
    constexpr int T = W / 8;
    uint32_t R[16];
#pragma unroll
    for (int u = 0; u < 16; u++) R[u] = 0u;
    uint32_t cx = 0u;
    stk = 0u;
    plast = 0u;
    uint4 nxt = tm_lds4(al);
#pragma unroll
    for (int j = 0; j < T; j++) {
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const uint4 a4 = nxt;
            if (8 * j + 4 * h + 4 < W) nxt = tm_lds4(al + 8 * j + 4 * h + 4);
            constexpr bool kWide = W <= 32;   // measured: wide rows faster at 512 / 1024 bits, spill at 2048
            if (h == 0) {
                tm_mad_row<0, kWide>(R, a4.x, bl);
                tm_mad_row<1, kWide>(R, a4.y, bl);
                tm_mad_row<2, kWide>(R, a4.z, bl);
                tm_mad_row<3, kWide>(R, a4.w, bl);
            } else {
                tm_mad_row<4, kWide>(R, a4.x, bl);
                tm_mad_row<5, kWide>(R, a4.y, bl);
                tm_mad_row<6, kWide>(R, a4.z, bl);
                tm_mad_row<7, kWide>(R, a4.w, bl);
            }
        }
        uint32_t in[8];
#pragma unroll
        for (int u = 0; u < 8; u++) in[u] = tm.above(R[u]);
        if (j < T - 1) {
#pragma unroll
            for (int u = 0; u < 8; u++) stk |= R[u];
        } else {
#pragma unroll
            for (int u = 0; u < 7; u++) stk |= R[u];
            plast = R[7];
        }
        tm_add_in(R + 8, in, cx);
        if (j < T - 1) {
#pragma unroll
            for (int u = 0; u < 8; u++) {
                R[u] = R[u + 8];
                R[u + 8] = 0u;
            }
        }
    }
    // R[8 .. 15] holds this lane's limbs of the high half with the carry cx
    // still owed to the lane above: add each lane's carry from below, then
    // resolve the carries that run on through all-ones lanes
#pragma unroll
    for (int u = 0; u < 8; u++) H[u] = R[u + 8];
    const uint32_t cin = tm.below(cx);
    const uint32_t g = tm_add_small(H, cin);     // g = 1 leaves H = 0: never both g and all ones
    if (__any_sync(kWarpAll, g != 0u)) (void)tm_add_small(H, tm.carry_in(g != 0u, tm_all_ones(H)));
}

// A team value: exponent and flags (bit0 sign, bit1 zero) replicated, this
// lane's 8 limbs.
struct TV {
    int e;
    unsigned f;
    uint32_t m[8];
};

template <int T>
__device__ __forceinline__ void tm_set_zero(TV& r, unsigned sign) {
    r.e = 0;
    r.f = 2u | (sign & 1u);
#pragma unroll
    for (int u = 0; u < 8; u++) r.m[u] = 0u;
}

// r = RN_p(a * b) with a given by its staged element in shared memory (`ar`:
// exponent, flags, two pad words, W limbs) and b by exponent, flags and this
// lane's limbs; the same result and the same status bits as mp_mul_acc.
template <int W>
__device__ __forceinline__ void tm_mul(const uint32_t* ar, int be, unsigned bf, const uint32_t (&bl)[8],
                                       const Team<W / 8>& tm, TV& r, unsigned& status) {
    constexpr int T = W / 8;
    const int ae = (int)ar[0];
    const unsigned af = ar[1];
    uint32_t H[8], plast, stk;
    tm_mul_full<W>(ar + 4, bl, tm, H, plast, stk);
    // P in [2^(2p-2), 2^(2p)): M = the top p bits after a shift of 0 or 1
    const uint32_t top = tm.from(H[7], T - 1);
    const int sh = (top >> 31) ? 0 : 1;
    uint32_t lo = tm.below(H[7]);
    if (tm.t == 0) lo = plast;
    uint32_t M[8];
    M[0] = __funnelshift_l(lo, H[0], sh);
#pragma unroll
    for (int u = 1; u < 8; u++) M[u] = __funnelshift_l(H[u - 1], H[u], sh);
    const uint32_t below = plast << sh;   // bits under M (lane 0), top bit = round bit
    const uint32_t rb = below >> 31;
    const uint32_t st = (below << 1) | stk;
    const uint32_t inc = tm.from((rb && (st != 0u || (M[0] & 1u))) ? 1u : 0u, 0);
    const uint32_t cout = tm_increment<T>(M, tm.t == 0 ? inc : 0u, tm);
    if (cout && tm.t == T - 1) M[7] = 0x80000000u;   // M was all ones: 2^p -> 2^(p-1), e + 1
    const unsigned sign = (af ^ bf) & 1u;
    if ((af | bf) & 2u) {
        tm_set_zero<T>(r, sign);
        return;
    }
    const long long e = (long long)ae + be - sh + (long long)cout;
    r.e = clamp_exp(e, status);
    r.f = sign;
#pragma unroll
    for (int u = 0; u < 8; u++) r.m[u] = M[u];
}


// r = RN_p(a + b), the team form of mp_add: the same frame [guard | W limbs
// | carry limb], here lane 0's extra guard limb, every lane's 8 limbs and the
// top lane's extra carry limb; the same alignment, carry chain, negation,
// normalisation and rounding, the same special cases and status bits.
template <int W>
__device__ __forceinline__ void tm_add(const TV& a, const TV& b, TV& r, const Team<W / 8>& tm, unsigned& status) {
    constexpr int T = W / 8;
    constexpr int p = 32 * W;
    // A zero operand (M = 0) becomes y, aligned by p + 2 bits: the sum is
    // then x exactly, which is mp_add's result (the other operand); two
    // zeros only differ from it in the sign, fixed at the end.
    const bool za = (a.f & 2u) != 0u, zb = (b.f & 2u) != 0u;
    const bool sw = za || (!zb && b.e > a.e);
    const int ex = sw ? b.e : a.e;
    const unsigned sx = (sw ? b.f : a.f) & 1u, sy = (sw ? a.f : b.f) & 1u;
    const long long dl = (long long)ex - (sw ? a.e : b.e);
    const int d = (za || zb || dl >= p + 2) ? p + 2 : (int)dl;
    uint32_t X[8], Y[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
        X[u] = sw ? b.m[u] : a.m[u];
        Y[u] = (za || zb) ? 0u : (sw ? a.m[u] : b.m[u]);
    }

    // Align y: limb k of the aligned value is funnel_r(y_(k+q), y_(k+q+1), r)
    // for k = -1 (the guard) .. W - 1, y_(-1) = 0 and y_(>= W) = 0; what
    // falls below the guard (limbs below q - 1, the low r bits of limb q - 1)
    // is sticky.  With d < 32 in every team of the warp only the neighbours'
    // edge limbs are needed and nothing falls below the guard.
    const int q = d >> 5, rs = d & 31;
    uint32_t w[10];
    bool stk = false;
    if (__all_sync(kWarpAll, q == 0)) {
        w[0] = tm.below(Y[7]);
#pragma unroll
        for (int u = 0; u < 8; u++) w[u + 1] = Y[u];
        w[9] = tm.above(Y[0]);
    } else {
        tm_window<T>(Y, 0u, q - 1, tm, w);
        uint32_t drop = 0u;
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int k = 8 * tm.t + u;
            drop |= k < q - 1 ? Y[u] : ((k == q - 1 && rs != 0) ? (Y[u] << (32 - rs)) : 0u);
        }
        stk = tm.any(drop != 0u);
    }

    // S = X + (Y xor mask) + (sub && !stk) over the frame, as in mp_add.
    // This lane's part of the chain: [guard (lane 0: 0 + y's guard, carry in
    // sub && !stk; other lanes 0 + 0), its 8 limbs, carry limb (top lane:
    // 0 + mask; other lanes 0 + 0, i.e. the carry out of its limbs)]; the
    // carries between lanes come from the look-ahead.
    const bool sub = sx != sy;
    const uint32_t mask = sub ? 0xFFFFFFFFu : 0u;
    uint32_t SG = tm.t == 0 ? (__funnelshift_r(w[0], w[1], rs) ^ mask) : 0u;
    uint32_t S[8];
#pragma unroll
    for (int u = 0; u < 8; u++) S[u] = __funnelshift_r(w[u + 1], w[u + 2], rs) ^ mask;
    uint32_t SC = tm.t == T - 1 ? mask : 0u;
    const uint32_t ci = (tm.t == 0 && sub && !stk) ? 1u : 0u;
    uint32_t co;
    asm("{\n\t.reg .u32 t;\n\t"
        "add.cc.u32 t, %11, 0xFFFFFFFF;\n\t"
        "addc.cc.u32 %0, %0, 0;\n\t"
        "addc.cc.u32 %1, %1, %12;\n\t"
        "addc.cc.u32 %2, %2, %13;\n\t"
        "addc.cc.u32 %3, %3, %14;\n\t"
        "addc.cc.u32 %4, %4, %15;\n\t"
        "addc.cc.u32 %5, %5, %16;\n\t"
        "addc.cc.u32 %6, %6, %17;\n\t"
        "addc.cc.u32 %7, %7, %18;\n\t"
        "addc.cc.u32 %8, %8, %19;\n\t"
        "addc.cc.u32 %9, %9, 0;\n\t"
        "addc.u32 %10, 0, 0;\n\t}"
        : "+r"(SG), "+r"(S[0]), "+r"(S[1]), "+r"(S[2]), "+r"(S[3]), "+r"(S[4]), "+r"(S[5]), "+r"(S[6]),
          "+r"(S[7]), "+r"(SC), "=r"(co)
        : "r"(ci), "r"(X[0]), "r"(X[1]), "r"(X[2]), "r"(X[3]), "r"(X[4]), "r"(X[5]), "r"(X[6]), "r"(X[7]));
    {
        const uint32_t k = tm.carry_in(tm.t < T - 1 && SC != 0u, tm_all_ones(S));
        asm("add.cc.u32 %0, %0, %10;\n\t"
            "addc.cc.u32 %1, %1, 0;\n\t"
            "addc.cc.u32 %2, %2, 0;\n\t"
            "addc.cc.u32 %3, %3, 0;\n\t"
            "addc.cc.u32 %4, %4, 0;\n\t"
            "addc.cc.u32 %5, %5, 0;\n\t"
            "addc.cc.u32 %6, %6, 0;\n\t"
            "addc.cc.u32 %7, %7, 0;\n\t"
            "addc.cc.u32 %8, %8, 0;\n\t"
            "addc.u32 %9, %9, 0;"
            : "+r"(S[0]), "+r"(S[1]), "+r"(S[2]), "+r"(S[3]), "+r"(S[4]), "+r"(S[5]), "+r"(S[6]), "+r"(S[7]),
              "+r"(SC), "+r"(co)
            : "r"(k));
    }
    const uint32_t cout = tm.from(co, T - 1);   // the frame's carry out (top lane's)
    unsigned sign = sx;
    const bool neg = sub && !cout;   // a borrow: only when d == 0 and My > Mx (exact): negate
    if (__any_sync(kWarpAll, neg)) {
        uint32_t NG = ~SG, N[8], NC = ~SC;
#pragma unroll
        for (int u = 0; u < 8; u++) N[u] = ~S[u];
        const uint32_t one = tm.t == 0 ? 1u : 0u;
        uint32_t g;
        asm("add.cc.u32 %0, %0, %10;\n\t"
            "addc.cc.u32 %1, %1, 0;\n\t"
            "addc.cc.u32 %2, %2, 0;\n\t"
            "addc.cc.u32 %3, %3, 0;\n\t"
            "addc.cc.u32 %4, %4, 0;\n\t"
            "addc.cc.u32 %5, %5, 0;\n\t"
            "addc.cc.u32 %6, %6, 0;\n\t"
            "addc.cc.u32 %7, %7, 0;\n\t"
            "addc.cc.u32 %8, %8, 0;\n\t"
            "addc.u32 %9, 0, 0;"
            : "+r"(NG), "+r"(N[0]), "+r"(N[1]), "+r"(N[2]), "+r"(N[3]), "+r"(N[4]), "+r"(N[5]), "+r"(N[6]),
              "+r"(N[7]), "=r"(g)
            : "r"(one));
        const uint32_t k = tm.carry_in(g != 0u, tm_all_ones(N));
        const uint32_t c2 = tm_add_small(N, k);
        NC += c2;
        if (neg) {
            SG = NG;
#pragma unroll
            for (int u = 0; u < 8; u++) S[u] = N[u];
            SC = NC;
            sign = sy;
        }
    }
    const uint32_t loc = (S[0] | S[1] | S[2] | S[3] | S[4] | S[5] | S[6] | S[7]) | (tm.t == 0 ? SG : 0u) |
                         (tm.t == T - 1 ? SC : 0u);
    const bool nz = tm.any(loc != 0u);

    // normalise: (A) a carry into the carry limb: one bit right; (B) the
    // leading bit in the top limb's two high bits: 0 or 1 bit left; (C) a
    // cancellation of leading bits (only with d <= 1, the sum then exact):
    // left by the leading-zero count
    const uint32_t SCt = tm.from(SC, T - 1);
    const uint32_t top = tm.from(S[7], T - 1);
    const bool caseA = SCt != 0u;
    const bool caseB = !caseA && (top >> 30) != 0u;
    const int s1 = (top >> 31) ? 0 : 1;
    uint32_t hi = tm.above(S[0]);
    if (tm.t == T - 1) hi = SC;
    uint32_t lo = tm.below(S[7]);
    if (tm.t == 0) lo = SG;
    uint32_t G, M[8];
    long long e;
    uint32_t sticky = 0u;
    if (caseA) {
        sticky = SG & 1u;
        G = __funnelshift_r(SG, S[0], 1);
#pragma unroll
        for (int u = 0; u < 7; u++) M[u] = __funnelshift_r(S[u], S[u + 1], 1);
        M[7] = __funnelshift_r(S[7], hi, 1);
        e = (long long)ex + 1;
    } else {
        G = SG << s1;
        M[0] = __funnelshift_l(lo, S[0], s1);
#pragma unroll
        for (int u = 1; u < 8; u++) M[u] = __funnelshift_l(S[u - 1], S[u], s1);
        e = (long long)ex - s1;
    }
    const bool caseC = !caseA && !caseB && nz;
    if (__any_sync(kWarpAll, caseC)) {
        int Lloc = 0;
#pragma unroll
        for (int u = 0; u < 8; u++)
            if (S[u]) Lloc = 32 * (8 * tm.t + 1 + u) + 32 - __clz(S[u]);
        if (tm.t == 0 && Lloc == 0 && SG) Lloc = 32 - __clz(SG);
        const unsigned bal = __ballot_sync(kWarpAll, Lloc != 0) & tm.bits();
        const int hl = bal ? 31 - __clz(bal) : tm.base;
        const int L = __shfl_sync(kWarpAll, Lloc, hl);
        const int sl = caseC ? 32 * (W + 1) - L : 0;
        const int qq = sl >> 5, rr = sl & 31;
        uint32_t wl[10];
        tm_window<T>(S, tm.from(SG, 0), -qq - 2, tm, wl);
        if (caseC) {
            G = __funnelshift_l(wl[0], wl[1], rr);
#pragma unroll
            for (int u = 0; u < 8; u++) M[u] = __funnelshift_l(wl[u + 1], wl[u + 2], rr);
            e = (long long)ex - sl;
        }
    }

    // round to nearest even on the guard (lane 0)
    const uint32_t rb = G >> 31;
    const uint32_t st = (G << 1) | sticky | (stk ? 1u : 0u);
    const uint32_t inc = tm.from((rb && (st != 0u || (M[0] & 1u))) ? 1u : 0u, 0);
    const uint32_t c3 = tm_increment<T>(M, tm.t == 0 ? inc : 0u, tm);
    if (c3 && tm.t == T - 1) M[7] = 0x80000000u;
    e += (long long)c3;

    if (!nz) {   // two zeros, or an exact cancellation (+0)
        tm_set_zero<T>(r, (za && zb) ? (a.f & b.f & 1u) : 0u);
        return;
    }
    r.e = clamp_exp(e, status);
    r.f = sign;
#pragma unroll
    for (int u = 0; u < 8; u++) r.m[u] = M[u];
}

}  // namespace mpg
