// Multi-limb block GEMM (Eq 2) with warp-cooperative values (mp_team.cuh):
// each output c_ij is held by a team of W / 8 lanes, 8 limbs per lane, for
// 512-, 1024- and 2048-bit formats.  The per-element operation sequence is
// that of Eq 1 (c = +0; for k = 1..l: c = RN(c + RN(a_ik b_kj)), k
// ascending), so the result is bit-identical to the one-thread-per-output
// kernels and to the definition.
//
// CTA: 256 threads = 256 / T teams = a BR x BC block of C; A rows and B
// columns are staged KT elements deep through shared memory, each element as
// [exponent, flags, pad, pad, W limbs] (16-byte aligned limbs): a team reads
// a's limbs four at a time (one address for the whole team: a broadcast) and
// each lane its own 8 limbs of b.
#include "common.cuh"
#include "kernels.h"
#include "mp_team.cuh"

namespace mpg {

template <int W>
struct TeamTile;
template <>
struct TeamTile<16> {   // 2 lanes per output
    static constexpr int BR = 8, BC = 16;
};
template <>
struct TeamTile<32> {   // 4 lanes per output
    static constexpr int BR = 8, BC = 8;
};
template <>
struct TeamTile<64> {   // 8 lanes per output
    static constexpr int BR = 4, BC = 8;
};

constexpr int kTeamKT = 8;

// Resident CTAs per SM the register budget is sized for: 80 / 128 / 128
// registers at 512 / 1024 / 2048 bits, none spilled (more resident CTAs,
// with spills, measured slower).
template <int W>
constexpr int team_min_ctas() {
    return W == 16 ? 3 : 2;
}

template <int W, int KT>
__global__ void __launch_bounds__(256, team_min_ctas<W>()) k_mp_team(int64_t m, int64_t l, int64_t n, View<const uint32_t> A,
                                                 View<const uint32_t> B, View<uint32_t> C, unsigned G,
                                                 unsigned* status) {
    constexpr int T = W / 8, BR = TeamTile<W>::BR, BC = TeamTile<W>::BC, E = W + 4;
    static_assert(BR * BC * T == 256, "one team per output, 256 threads");
    __shared__ __align__(16) uint32_t sm[(BR + BC) * KT * E];
    auto As = reinterpret_cast<uint32_t (*)[BR][E]>(sm);            // [k][row][word]
    auto Bs = reinterpret_cast<uint32_t (*)[BC][E]>(sm + KT * BR * E);
    const Team<T> tm;
    const int team = (int)threadIdx.x / T;
    const int ty = team / BC, tx = team % BC;
    const unsigned tiles_m = ceil_div(m, BR), tiles_n = ceil_div(n, BC);
    unsigned ti, tj;
    raster(blockIdx.x, tiles_m, tiles_n, G, ti, tj);
    const int64_t i0 = (int64_t)ti * BR, j0 = (int64_t)tj * BC, z = blockIdx.y;
    TV c;
    tm_set_zero<T>(c, 0u);
    unsigned st = 0u;
    for (int64_t k0 = 0; k0 < l; k0 += KT) {
        // planes in word order: exponent, flags, then the limbs from word 4;
        // entries outside the matrices are zeros (flags 2)
        for (int idx = threadIdx.x; idx < (2 + W) * BR * KT; idx += 256) {
            const int q = idx / (BR * KT), rem = idx % (BR * KT);
            const int r = rem / KT, cc = rem % KT;
            const int64_t i = i0 + r, k = k0 + cc;
            As[cc][r][q < 2 ? q : q + 2] = (i < m && k < l) ? A.load(A.at(z, q, i, k)) : (q == 1 ? 2u : 0u);
        }
        for (int idx = threadIdx.x; idx < (2 + W) * KT * BC; idx += 256) {
            const int q = idx / (KT * BC), rem = idx % (KT * BC);
            const int rb = rem / BC, cb = rem % BC;
            const int64_t k = k0 + rb, j = j0 + cb;
            Bs[rb][cb][q < 2 ? q : q + 2] = (k < l && j < n) ? B.load(B.at(z, q, k, j)) : (q == 1 ? 2u : 0u);
        }
        __syncthreads();
        const int kmax = (l - k0) < KT ? (int)(l - k0) : KT;
        for (int kk = 0; kk < kmax; kk++) {
            const uint32_t* ar = &As[kk][ty][0];
            const uint32_t* br = &Bs[kk][tx][0];
            const uint4 b0 = *reinterpret_cast<const uint4*>(br + 4 + 8 * tm.t);
            const uint4 b1 = *reinterpret_cast<const uint4*>(br + 8 + 8 * tm.t);
            const uint32_t bl[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
            TV t;
            tm_mul<W>(ar, (int)br[0], br[1], bl, tm, t, st);
            tm_add<W>(c, t, c, tm, st);
        }
        __syncthreads();
    }
    const int64_t i = i0 + ty, j = j0 + tx;
    if (i < m && j < n) {
        uint32_t* p = C.at(z, 0, i, j);
        if (tm.t == 0) {
            C.store(p, (uint32_t)c.e);
            C.store(p + C.ps, c.f);
        }
#pragma unroll
        for (int u = 0; u < 8; u++) C.store(p + (2 + 8 * tm.t + u) * C.ps, c.m[u]);
    }
    if (st) atomicOr(status, st);
}

template <int W>
static void launch_team(int64_t m, int64_t l, int64_t n, int64_t batch, View<const uint32_t> A,
                        View<const uint32_t> B, View<uint32_t> C, int n_min, unsigned* status, cudaStream_t s) {
    constexpr int BR = TeamTile<W>::BR, BC = TeamTile<W>::BC;
    const unsigned G = n_min > BR ? (unsigned)(n_min / BR) : 1u;
    dim3 grd(ceil_div(m, BR) * ceil_div(n, BC), (unsigned)batch);
    k_mp_team<W, kTeamKT><<<grd, 256, 0, s>>>(m, l, n, A, B, C, G, status);
}

// Which block kernel multi-limb GEMMs of w limbs use: 1 = one thread per
// output (gemm_mp.cu), 2 = a team of w / 8 lanes per output (above), 0 = the
// default: the team kernel when the one-thread kernel's grid (16 x 16
// outputs per CTA) would have at most one CTA for every two SMs.  A team
// computes the full W^2 limb product where the one-thread kernel forms the
// high half first, so with both grids filling the GPU the team kernel
// reaches 0.56 / 0.56 / 0.77 of its throughput at 512 / 1024 / 2048 bits;
// with few outputs (small m x n, any l) it spreads each output over W / 8
// lanes and 4-8x more CTAs and is 1.1-1.2x / 1.2-2.1x / 1.4-4.9x faster
// (block GEMMs of 16^2 to 128^2 outputs, l = 32 to 4096, on GB300).
static int g_mp_leaf = 0;

static int leaf_choice(int w, int64_t m, int64_t n, int64_t batch, int sms) {
    if (w != 16 && w != 32 && w != 64) return MPGEMM_MP_LEAF_THREAD;
    if (g_mp_leaf != MPGEMM_MP_LEAF_DEFAULT) return g_mp_leaf;
    const int64_t thread_ctas = (int64_t)ceil_div(m, 16) * ceil_div(n, 16) * batch;
    return 2 * thread_ctas <= sms ? MPGEMM_MP_LEAF_TEAM : MPGEMM_MP_LEAF_THREAD;
}

bool mp_team_leaf(int w, int64_t m, int64_t n, int64_t batch, cudaStream_t s) {
    if (w != 16 && w != 32 && w != 64) return false;
    if (g_mp_leaf != MPGEMM_MP_LEAF_DEFAULT) return g_mp_leaf == MPGEMM_MP_LEAF_TEAM;
    return leaf_choice(w, m, n, batch, stream_sms(s)) == MPGEMM_MP_LEAF_TEAM;
}

int mp_gemm_team(int w, int64_t m, int64_t l, int64_t n, int64_t batch, View<const uint32_t> A,
                 View<const uint32_t> B, View<uint32_t> C, int n_min, unsigned* status, cudaStream_t s) {
    switch (w) {
        case 16: launch_team<16>(m, l, n, batch, A, B, C, n_min, status, s); break;
        case 32: launch_team<32>(m, l, n, batch, A, B, C, n_min, status, s); break;
        case 64: launch_team<64>(m, l, n, batch, A, B, C, n_min, status, s); break;
        default: return MPGEMM_EUNSUPPORTED;
    }
    return MPGEMM_OK;
}

}  // namespace mpg

extern "C" int mpgemm_mp_leaf_choice(int prec_bits, int64_t m, int64_t n, int64_t batch, int sms) {
    if (prec_bits <= 0 || prec_bits % 32 || m < 0 || n < 0 || batch < 1 || sms < 1) return MPGEMM_EINVAL;
    return mpg::leaf_choice(prec_bits / 32, m, n, batch, sms);
}

extern "C" int mpgemm_set_mp_leaf(int leaf) {
    if (leaf < 0 || leaf > 2) return MPGEMM_EINVAL;
    const int prev = mpg::g_mp_leaf;
    mpg::g_mp_leaf = leaf;
    return prev;
}
