// Multi-limb GEMM kernels (simple, Eq 1, and block, Eq 2) and the
// elementwise add/sub used by Strassen (Eq 3), for p = 32 W bits.
//
// Both GEMM kernels keep the per-element operation sequence of Eq 1
// (c = +0; for k = 1..l: c = RN(c + RN(a_ik b_kj))), so they are
// bit-identical to each other and to the definition.  The work is on the
// integer pipe (W^2 32x32->64 multiplies per product plus O(W) alignment and
// rounding), one thread per output.
#include "common.cuh"
#include "kernels.h"
#include "mp_arith.cuh"
#include "tiles.cuh"
#include "profile.h"

namespace mpg {

template <int W, bool CLOSE>
__global__ void __launch_bounds__(256) k_mp_simple(int64_t m, int64_t l, int64_t n, View<const uint32_t> A,
                                                   View<const uint32_t> B, View<uint32_t> C, unsigned* status) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = (int64_t)blockIdx.y * blockDim.y + threadIdx.y;
    int64_t z = blockIdx.z;
    if (i >= m || j >= n) return;
    unsigned st = 0u;
    MPV<W> c;
    mp_set_zero(c, 0u);
    for (int64_t k = 0; k < l; k++) {
        MPV<W> a, b;
        load_mp(a, A, A.at(z, 0, i, k));
        load_mp(b, B, B.at(z, 0, k, j));
        mp_mac<W, CLOSE>(c, a, b, st);
    }
    store_mp(c, C, C.at(z, 0, i, j));
    if (st) atomicOr(status, st);
}

// Resident CTAs per SM the block kernel's register budget is sized for
// (0: the compiler's choice).  With their operands streamed from shared
// memory, 512- and 1024-bit tiles fit 3 and 2 CTAs per SM.
template <int W>
constexpr int mp_block_min_ctas() {
    return W == 16 ? 3 : W == 32 ? 2 : W == 64 ? 1 : 0;
}

// CTA = 16 x 16 outputs (mp_block_tile); CTA order follows the super-tile
// raster with group G.
template <int W, int KT, bool CLOSE>
__global__ void __launch_bounds__(256, mp_block_min_ctas<W>()) k_mp_block(int64_t m, int64_t l, int64_t n, View<const uint32_t> A,
                                                  View<const uint32_t> B, View<uint32_t> C, unsigned G,
                                                  unsigned* status) {
    constexpr int BM = 16;
    __shared__ __align__(16) uint32_t sm[mp_tile_words<W, KT>()];
    const unsigned tiles_m = ceil_div(m, BM), tiles_n = ceil_div(n, BM);
    unsigned tm, tn;
    raster(blockIdx.x, tiles_m, tiles_n, G, tm, tn);
    unsigned st = 0u;
    mp_block_tile<W, KT, CLOSE>(m, l, n, A, B, C, blockIdx.y, (int64_t)tm * BM, (int64_t)tn * BM, sm, st);
    if (st) atomicOr(status, st);
}

template <int W>
__global__ void k_mp_addsub(int64_t r, int64_t c, View<uint32_t> Z, View<const uint32_t> X, View<const uint32_t> Y,
                            int sub, unsigned* status) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = (int64_t)blockIdx.y;
    int64_t z = blockIdx.z;
    if (j >= c) return;
    unsigned st = 0u;
    MPV<W> x, y, s;
    load_mp(x, X, X.at(z, 0, i, j));
    load_mp(y, Y, Y.at(z, 0, i, j));
    if (sub) y.f ^= 1u;
    mp_add<W>(x, y, s, st);
    store_mp(s, Z, Z.at(z, 0, i, j));
    if (st) atomicOr(status, st);
}

// Operands of similar magnitude (set by the integer pipe's DD / QD
// conversions around their GEMMs): the kernels with mp_add's alignment
// shortcut (widths 2 to 16, the integer pipe's).
static thread_local bool t_close_operands = false;

CloseOperandsScope::CloseOperandsScope() : prev_(t_close_operands) { t_close_operands = true; }
CloseOperandsScope::~CloseOperandsScope() { t_close_operands = prev_; }

template <int W, bool CLOSE>
static void launch_mp(int algo, int64_t m, int64_t l, int64_t n, int64_t batch, View<const uint32_t> A,
                      View<const uint32_t> B, View<uint32_t> C, int n_min, unsigned* status, cudaStream_t s) {
    if (algo == MPGEMM_SIMPLE) {
        dim3 blk(16, 16);
        dim3 grd(ceil_div(n, 16), ceil_div(m, 16), (unsigned)batch);
        k_mp_simple<W, CLOSE><<<grd, blk, 0, s>>>(m, l, n, A, B, C, status);
    } else {
        unsigned G = n_min > 16 ? (unsigned)(n_min / 16) : 1u;
        dim3 grd(ceil_div(m, 16) * ceil_div(n, 16), (unsigned)batch);
        constexpr int KT = W >= 16 ? 4 : 8;
        k_mp_block<W, KT, CLOSE><<<grd, 256, 0, s>>>(m, l, n, A, B, C, G, status);
    }
}

template <int W>
static int mp_gemm_w(int algo, int64_t m, int64_t l, int64_t n, int64_t batch, View<const uint32_t> A,
                     View<const uint32_t> B, View<uint32_t> C, int n_min, cudaStream_t s) {
    unsigned* status = device_status_ptr();
    if (!status) return MPGEMM_ECUDA;
    ProfScope ps(s);
    if (algo != MPGEMM_SIMPLE && mp_team_leaf(W, m, n, batch, s)) {
        const int rc = mp_gemm_team(W, m, l, n, batch, A, B, C, n_min, status, s);
        if (rc != MPGEMM_OK) return rc;
    } else if constexpr (W >= 2 && W <= 16) {
        if (t_close_operands) launch_mp<W, true>(algo, m, l, n, batch, A, B, C, n_min, status, s);
        else launch_mp<W, false>(algo, m, l, n, batch, A, B, C, n_min, status, s);
    } else {
        launch_mp<W, false>(algo, m, l, n, batch, A, B, C, n_min, status, s);
    }
    return check_launch();
}

int mp_gemm(int w, int algo, int64_t m, int64_t l, int64_t n, int64_t batch, View<const uint32_t> A,
            View<const uint32_t> B, View<uint32_t> C, int n_min, cudaStream_t s) {
    if (m == 0 || n == 0 || batch == 0) return MPGEMM_OK;
    switch (w) {
        case 1: return mp_gemm_w<1>(algo, m, l, n, batch, A, B, C, n_min, s);
        case 2: return mp_gemm_w<2>(algo, m, l, n, batch, A, B, C, n_min, s);
        case 4: return mp_gemm_w<4>(algo, m, l, n, batch, A, B, C, n_min, s);
        case 8: return mp_gemm_w<8>(algo, m, l, n, batch, A, B, C, n_min, s);
        case 16: return mp_gemm_w<16>(algo, m, l, n, batch, A, B, C, n_min, s);
        case 32: return mp_gemm_w<32>(algo, m, l, n, batch, A, B, C, n_min, s);
        case 64: return mp_gemm_w<64>(algo, m, l, n, batch, A, B, C, n_min, s);
        default: return MPGEMM_EUNSUPPORTED;
    }
}

template <int W>
static int mp_addsub_w(int64_t r, int64_t c, int64_t batch, View<uint32_t> Z, View<const uint32_t> X,
                       View<const uint32_t> Y, int sub, cudaStream_t s) {
    unsigned* status = device_status_ptr();
    if (!status) return MPGEMM_ECUDA;
    dim3 grd(ceil_div(c, 128), (unsigned)r, (unsigned)batch);
    k_mp_addsub<W><<<grd, 128, 0, s>>>(r, c, Z, X, Y, sub, status);
    return check_launch();
}

int mp_addsub(int w, int64_t r, int64_t c, int64_t batch, View<uint32_t> Z, View<const uint32_t> X,
              View<const uint32_t> Y, int sub, cudaStream_t s) {
    if (r == 0 || c == 0 || batch == 0) return MPGEMM_OK;
    switch (w) {
        case 1: return mp_addsub_w<1>(r, c, batch, Z, X, Y, sub, s);
        case 2: return mp_addsub_w<2>(r, c, batch, Z, X, Y, sub, s);
        case 4: return mp_addsub_w<4>(r, c, batch, Z, X, Y, sub, s);
        case 8: return mp_addsub_w<8>(r, c, batch, Z, X, Y, sub, s);
        case 16: return mp_addsub_w<16>(r, c, batch, Z, X, Y, sub, s);
        case 32: return mp_addsub_w<32>(r, c, batch, Z, X, Y, sub, s);
        case 64: return mp_addsub_w<64>(r, c, batch, Z, X, Y, sub, s);
        default: return MPGEMM_EUNSUPPORTED;
    }
}

}  // namespace mpg
