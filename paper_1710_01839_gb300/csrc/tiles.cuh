// Device building blocks shared by the GEMM kernels and the batched
// persistent kernel: the DD / QD element formats and one CTA's block of C.
#pragma once

#include "common.cuh"
#include "ddqd.cuh"
#include "mp_arith.cuh"

namespace mpg {

struct DDFmt {
    static constexpr int P = 2;
    static constexpr int R = DD_RENORM;
    using Acc = DDAcc;
    __device__ static void zero(Acc& c) { dd_zero(c); }
    __device__ static void mac(Acc& c, const double* a, const double* b) { dd_mac(c, a[0], a[1], b[0], b[1]); }
    __device__ static void renorm(Acc& c) { dd_renorm(c); }
    __device__ static void finish(Acc& c, double* out) {
        double h, l;
        two_sum(c.s, c.t, h, l);
        out[0] = h;
        out[1] = l;
    }
};

struct QDFmt {
    static constexpr int P = 4;
    static constexpr int R = QD_RENORM;
    using Acc = QDAcc;
    __device__ static void zero(Acc& c) { qd_zero(c); }
    __device__ static void mac(Acc& c, const double* a, const double* b) { qd_mac(c, a, b); }
    __device__ static void renorm(Acc& c) { qd_renorm(c); }
    __device__ static void finish(Acc& c, double* out) {
        qd_finish(c);
        out[0] = c.s0;
        out[1] = c.s1;
        out[2] = c.s2;
        out[3] = c.s3;
    }
};

// Shared memory (doubles) of one ddqd_block_tile: two KT-deep panels, each
// k-plane P rows of BM values plus one pad.
template <class Fmt, int BM, int KT>
__host__ __device__ constexpr int ddqd_tile_doubles() {
    return 2 * KT * (BM * Fmt::P + 1);
}

// One BM x BM block of C (rows i0.., columns j0.., batch z) computed by the
// calling CTA (NT = (BM/RM)^2 threads): each thread an RM x RM register tile
// (rows ty + r*TPD, columns tx + c*TPD); K advances in panels of KT staged
// through shared memory `sm` (ddqd_tile_doubles() doubles) as [k][plane][row]
// with an odd k-stride of BM*P + 1 doubles: a warp's B reads are BM
// consecutive doubles (no bank conflict), its A reads broadcasts, and the
// padding spreads a panel store's k-planes over the banks.  The next panel's
// global loads are issued before the current panel's arithmetic.
template <class Fmt, int BM, int RM, int KT>
__device__ __forceinline__ void ddqd_block_tile(int64_t m, int64_t l, int64_t n, const View<const double>& A,
                                                const View<const double>& B, const View<double>& C, int64_t z,
                                                int64_t i0, int64_t j0, double* sm) {
    constexpr int P = Fmt::P;
    constexpr int TPD = BM / RM;
    constexpr int NT = TPD * TPD;
    constexpr int LD = (BM * KT) / NT;   // elements per thread per panel and operand
    static_assert((BM * KT) % NT == 0, "panel must split evenly over the threads");
    static_assert(KT % Fmt::R == 0, "renormalisation period must divide the panel depth");
    constexpr int KS = BM * P + 1;   // k-plane stride (doubles)
    double* As = sm;                 // element (k, plane q, row r) at k KS + q BM + r
    double* Bs = sm + KT * KS;       // element (k, plane q, column c) at k KS + q BM + c
    const int tid = threadIdx.x;
    const int ty = tid / TPD, tx = tid % TPD;

    typename Fmt::Acc acc[RM][RM];
#pragma unroll
    for (int r = 0; r < RM; r++)
#pragma unroll
        for (int c = 0; c < RM; c++) Fmt::zero(acc[r][c]);

    double ra[LD][P], rb[LD][P];
    auto gload = [&](int64_t k0) {
#pragma unroll
        for (int v = 0; v < LD; v++) {
            int idx = tid + v * NT;
            int r = idx / KT, c = idx % KT;          // A panel: BM rows x KT
            int64_t i = i0 + r, k = k0 + c;
            bool ok = i < m && k < l;
#pragma unroll
            for (int q = 0; q < P; q++) ra[v][q] = ok ? A.load(A.at(z, q, i, k)) : 0.0;
            int rr = idx / BM, cc = idx % BM;        // B panel: KT rows x BM
            int64_t kb = k0 + rr, j = j0 + cc;
            bool okb = kb < l && j < n;
#pragma unroll
            for (int q = 0; q < P; q++) rb[v][q] = okb ? B.load(B.at(z, q, kb, j)) : 0.0;
        }
    };
    auto sstore = [&]() {
#pragma unroll
        for (int v = 0; v < LD; v++) {
            int idx = tid + v * NT;
            int r = idx / KT, c = idx % KT;
            int rr = idx / BM, cc = idx % BM;
#pragma unroll
            for (int q = 0; q < P; q++) {
                As[c * KS + q * BM + r] = ra[v][q];
                Bs[rr * KS + q * BM + cc] = rb[v][q];
            }
        }
    };

    gload(0);
    sstore();
    __syncthreads();
    for (int64_t k0 = 0; k0 < l; k0 += KT) {
        const bool more = k0 + KT < l;
        if (more) gload(k0 + KT);
#pragma unroll
        for (int kk = 0; kk < KT; kk++) {
            double a[RM][P], b[RM][P];
#pragma unroll
            for (int r = 0; r < RM; r++)
#pragma unroll
                for (int q = 0; q < P; q++) a[r][q] = As[kk * KS + q * BM + ty + r * TPD];
#pragma unroll
            for (int c = 0; c < RM; c++)
#pragma unroll
                for (int q = 0; q < P; q++) b[c][q] = Bs[kk * KS + q * BM + tx + c * TPD];
#pragma unroll
            for (int r = 0; r < RM; r++)
#pragma unroll
                for (int c = 0; c < RM; c++) Fmt::mac(acc[r][c], a[r], b[c]);
            if ((kk + 1) % Fmt::R == 0) {
#pragma unroll
                for (int r = 0; r < RM; r++)
#pragma unroll
                    for (int c = 0; c < RM; c++) Fmt::renorm(acc[r][c]);
            }
        }
        __syncthreads();
        if (more) {
            sstore();
            __syncthreads();
        }
    }

#pragma unroll
    for (int r = 0; r < RM; r++)
#pragma unroll
        for (int c = 0; c < RM; c++) {
            int64_t i = i0 + ty + r * TPD, j = j0 + tx + c * TPD;
            double out[P];
            Fmt::finish(acc[r][c], out);
            if (i < m && j < n) {
#pragma unroll
                for (int q = 0; q < P; q++) C.store(C.at(z, q, i, j), out[q]);
            }
        }
}

template <int W>
__device__ __forceinline__ void load_mp(MPV<W>& v, const View<const uint32_t>& V, const uint32_t* p) {
    v.e = (int)V.load(p);
    v.f = V.load(p + V.ps);
MP_UNROLL
    for (int i = 0; i < W; i++) v.m[i] = V.load(p + (2 + i) * V.ps);
}

template <int W>
__device__ __forceinline__ void store_mp(const MPV<W>& v, const View<uint32_t>& V, uint32_t* p) {
    V.store(p, (uint32_t)v.e);
    V.store(p + V.ps, v.f);
MP_UNROLL
    for (int i = 0; i < W; i++) V.store(p + (2 + i) * V.ps, v.m[i]);
}

template <int W, bool CLOSE = false>
__device__ __forceinline__ void mp_mac(MPV<W>& c, const MPV<W>& a, const MPV<W>& b, unsigned& st) {
    MPV<W> t;
    mp_mul<W>(a, b, t, st);
    MPV<W> s;
    mp_add<W, CLOSE>(c, t, s, st);
    c = s;
}

// Operands of this width and up are not held in registers: the block
// kernel's multiply reads both from shared memory (fewer live registers, so
// more resident CTAs per SM).
constexpr int MP_STREAM_LIMBS = 16;

// Shared memory (words) of one mp_block_tile: two KT-deep panels of 16
// elements, each [exponent, flags, (pad, pad,) W limbs]; from 4 limbs up the
// limbs start at a 16-byte boundary, so an element is read with 128-bit
// loads (register operands) or streamed four limbs per load.
template <int W>
__host__ __device__ constexpr int mp_tile_limb_offset() {
    return W >= 4 ? 4 : 2;
}
template <int W, int KT>
__host__ __device__ constexpr int mp_tile_words() {
    return 2 * KT * 16 * (mp_tile_limb_offset<W>() + W);
}

// One 16 x 16 block of C (one output per thread, 256 threads) with A rows and
// B columns staged KT elements deep through shared memory `sm`
// (mp_tile_words<W, KT>() words, 16-byte aligned) as [k][row][word];
// device-side flags are ORed into `st`.  CLOSE: mp_add's alignment shortcut
// for operands of similar magnitude.
template <int W, int KT, bool CLOSE = false>
__device__ __forceinline__ void mp_block_tile(int64_t m, int64_t l, int64_t n, const View<const uint32_t>& A,
                                              const View<const uint32_t>& B, const View<uint32_t>& C, int64_t z,
                                              int64_t i0, int64_t j0, uint32_t* sm, unsigned& st) {
    constexpr int BM = 16;
    constexpr int OFF = mp_tile_limb_offset<W>();
    constexpr int E = OFF + W;            // words per staged element
    constexpr int WORDS = BM * KT * (2 + W);
    auto As = reinterpret_cast<uint32_t (*)[BM][E]>(sm);
    auto Bs = reinterpret_cast<uint32_t (*)[BM][E]>(sm + KT * BM * E);
    const int tid = threadIdx.x, ty = tid / BM, tx = tid % BM;
    MPV<W> c;
    mp_set_zero(c, 0u);
    // 128 / 256 bits (KT = 8): a panel holds 128 elements of A and 128 of B,
    // one per thread, staged whole: threads 0..127 take A's (row r, k offset
    // cc), rows fastest (consecutive threads write consecutive 16-byte
    // aligned elements: at most 2-way bank conflicts), threads 128..255 take
    // B's (k offset rb, column cb), columns fastest (coalesced reads).  The
    // element's address is formed once; per panel only k moves.
    constexpr bool kWhole = (W % 4 == 0) && (W < MP_STREAM_LIMBS) && (KT == 8) && (OFF == 4);
    const bool sA = tid < 128;
    const int el = tid & 127;
    const int er = sA ? (el & 15) : (el >> 4), ec = sA ? (el >> 4) : (el & 15);   // A: (r, cc); B: (rb, cb)
    const uint32_t* gbase = nullptr;
    bool fixed_ok = false;
    int64_t ps = 0;
    uint32_t* sdst = nullptr;
    if constexpr (kWhole) {
        if (sA) {
            fixed_ok = i0 + er < m;
            gbase = A.p + z * A.bs + (fixed_ok ? (i0 + er) * A.ld : 0);
            ps = A.ps;
            sdst = &As[ec][er][0];
        } else {
            fixed_ok = j0 + ec < n;
            gbase = B.p + z * B.bs + (fixed_ok ? j0 + ec : 0);
            ps = B.ps;
            sdst = &Bs[er][ec][0];
        }
    }
    for (int64_t k0 = 0; k0 < l; k0 += KT) {
        if constexpr (kWhole) {
            const int64_t k = k0 + (sA ? ec : er);
            const bool ok = fixed_ok && k < l;
            const uint32_t* src = gbase + (sA ? k : k * B.ld);
            const View<const uint32_t>& SV = sA ? A : B;
            uint32_t w[OFF + W];
            w[0] = ok ? SV.load(src) : 0u;
            w[1] = ok ? SV.load(src + ps) : 2u;   // flags: zero
            w[2] = 0u;
            w[3] = 0u;
MP_UNROLL
            for (int q = 0; q < W; q++) w[OFF + q] = ok ? SV.load(src + (2 + q) * ps) : 0u;
MP_UNROLL
            for (int q = 0; q < OFF + W; q += 4)
                *reinterpret_cast<uint4*>(sdst + q) = make_uint4(w[q], w[q + 1], w[q + 2], w[q + 3]);
        } else
        for (int idx = tid; idx < WORDS; idx += 256) {
            int q = idx / (BM * KT), rem = idx % (BM * KT);
            int slot = q < 2 ? q : q - 2 + OFF;
            int r = rem / KT, cc = rem % KT;          // A: row r, k = k0 + cc
            int64_t i = i0 + r, k = k0 + cc;
            uint32_t va = (i < m && k < l) ? A.load(A.at(z, q, i, k)) : (q == 1 ? 2u : 0u);
            As[cc][r][slot] = va;
            int rb = rem / BM, cb = rem % BM;         // B: k = k0 + rb, column cb
            int64_t kb = k0 + rb, j = j0 + cb;
            uint32_t vb = (kb < l && j < n) ? B.load(B.at(z, q, kb, j)) : (q == 1 ? 2u : 0u);
            Bs[rb][cb][slot] = vb;
        }
        __syncthreads();
        const int kmax = (l - k0) < KT ? (int)(l - k0) : KT;
        for (int kk = 0; kk < kmax; kk++) {
            const uint32_t* ar = &As[kk][ty][0];
            const uint32_t* br = &Bs[kk][tx][0];
            MPV<W> t;
            if constexpr (W >= MP_STREAM_LIMBS) {
                mp_mul_acc<W>((int)ar[0], ar[1], SmemLimbs{ar + OFF}, (int)br[0], br[1], SmemLimbs{br + OFF}, t, st);
            } else if constexpr (W % 4 == 0) {
                MPV<W> a, b;
                const uint2 ha = *reinterpret_cast<const uint2*>(ar), hb = *reinterpret_cast<const uint2*>(br);
                a.e = (int)ha.x;
                a.f = ha.y;
                b.e = (int)hb.x;
                b.f = hb.y;
MP_UNROLL
                for (int w = 0; w < W; w += 4) {
                    const uint4 va = *reinterpret_cast<const uint4*>(ar + OFF + w);
                    const uint4 vb = *reinterpret_cast<const uint4*>(br + OFF + w);
                    a.m[w] = va.x;
                    a.m[w + 1] = va.y;
                    a.m[w + 2] = va.z;
                    a.m[w + 3] = va.w;
                    b.m[w] = vb.x;
                    b.m[w + 1] = vb.y;
                    b.m[w + 2] = vb.z;
                    b.m[w + 3] = vb.w;
                }
                mp_mul<W>(a, b, t, st);
            } else {
                MPV<W> a, b;
                a.e = (int)ar[0];
                a.f = ar[1];
                b.e = (int)br[0];
                b.f = br[1];
MP_UNROLL
                for (int w = 0; w < W; w++) {
                    a.m[w] = ar[OFF + w];
                    b.m[w] = br[OFF + w];
                }
                mp_mul<W>(a, b, t, st);
            }
            MPV<W> s;
            mp_add<W, CLOSE>(c, t, s, st);
            c = s;
        }
        __syncthreads();
    }
    int64_t i = i0 + ty, j = j0 + tx;
    if (i < m && j < n) store_mp(c, C, C.at(z, 0, i, j));
}

}  // namespace mpg
