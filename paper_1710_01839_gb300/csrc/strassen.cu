// Strassen's algorithm (Eq 3), breadth first and batched.
//
// Level k (1..d) holds 7^k sub-problems of size (m/2^k, l/2^k, n/2^k).  For
// parent p and child c in 0..6 (P1..P7 of Eq 3):
//   A side: P1 A11+A22, P2 A21+A22, P3 A11, P4 A22, P5 A11+A12, P6 A21-A11,
//           P7 A12-A22
//   B side: P1 B11+B22, P2 B11, P3 B12-B22, P4 B21-B11, P5 B22, P6 B11+B12,
//           P7 B21+B22
// and the parent's product is assembled from its seven children as
//   C11 = ((P1 + P4) - P5) + P7, C12 = P3 + P5, C21 = P2 + P4,
//   C22 = ((P1 + P3) - P2) + P6,
// left to right, every add rounded in the format.  Leaves are the block
// algorithm (Eq 2) with block size n_min, all 7^d of them in one launch.
//
// Dimensions that 2^d does not divide: A and B are read as if extended with
// zero rows and columns to the next multiples of 2^d (the level-1 operand
// kernels return zero outside the caller's matrices, nothing is copied) and
// the level-1 assembly writes only the leading m x n block of C.
#include "common.cuh"
#include "ddqd.cuh"
#include "kernels.h"
#include "mp_arith.cuh"
#include "strassen.h"

namespace mpg {

// quadrant codes: q = 2*row_half + col_half (11 -> 0, 12 -> 1, 21 -> 2, 22 -> 3)
struct ChildOps {
    signed char qa[7], qb[7], op[7];   // op: 0 = copy qa, 1 = qa + qb, 2 = qa - qb
};

static ChildOps a_side_ops() {
    ChildOps o = {{0, 2, 0, 3, 0, 2, 1}, {3, 3, 0, 0, 1, 0, 3}, {1, 1, 0, 0, 1, 2, 2}};
    return o;
}
static ChildOps b_side_ops() {
    ChildOps o = {{0, 0, 1, 2, 3, 0, 2}, {3, 0, 3, 0, 0, 1, 3}, {1, 0, 2, 2, 0, 1, 1}};
    return o;
}

// The same tables at compile time (side 0: A, 1: B; what 0: qa, 1: qb, 2: op).
__host__ __device__ constexpr int child_op(int side, int what, int c) {
    constexpr signed char t[2][3][7] = {{{0, 2, 0, 3, 0, 2, 1}, {3, 3, 0, 0, 1, 0, 3}, {1, 1, 0, 0, 1, 2, 2}},
                                        {{0, 0, 1, 2, 3, 0, 2}, {3, 0, 3, 0, 0, 1, 3}, {1, 0, 2, 2, 0, 1, 1}}};
    return t[side][what][c];
}

// ---------------------------------------------------------------- element ops

// add: the sum rounded in the format (FP64 error terms); add_int: the same
// sum where `rare` stays false, with fewer FP64 operations (DD: three of the
// four error terms on the integer pipe, 8 FP64 operations instead of 10;
// QD: add itself); neg_int: -x for add_int's operands.
struct DDE {
    static constexpr int P = 2;
    __device__ static void add(const double* x, const double* y, double* z) { dd_add(x[0], x[1], y[0], y[1], z[0], z[1]); }
    __device__ static void add_int(const double* x, const double* y, double* z, bool& rare) {
        dd_add_int(x[0], x[1], y[0], y[1], z[0], z[1], rare);
    }
    __device__ static double neg_int(double v) { return neg_bits(v); }
};
struct QDE {
    static constexpr int P = 4;
    __device__ static void add(const double* x, const double* y, double* z) { qd_add(x, y, z); }
    __device__ static void add_int(const double* x, const double* y, double* z, bool&) { qd_add(x, y, z); }
    __device__ static double neg_int(double v) { return -v; }
};

template <class E>
__device__ __forceinline__ void ld(const View<const double>& V, int64_t z, int64_t i, int64_t j, double* x) {
#pragma unroll
    for (int q = 0; q < E::P; q++) x[q] = V.get(V.at(z, q, i, j));
}
template <class E>
__device__ __forceinline__ void st(const View<double>& V, int64_t z, int64_t i, int64_t j, const double* x) {
#pragma unroll
    for (int q = 0; q < E::P; q++) V.store(V.at(z, q, i, j), x[q]);
}
template <class E>
__device__ __forceinline__ void neg(double* x) {
#pragma unroll
    for (int q = 0; q < E::P; q++) x[q] = -x[q];
}

// Element (r, c) of parent p, zero outside its first xr rows and xc columns.
template <class E>
__device__ __forceinline__ void ld_ext(const View<const double>& V, int64_t p, int64_t r, int64_t c, int64_t xr,
                                       int64_t xc, double* x) {
    if (r < xr && c < xc) {
        ld<E>(V, p, r, c, x);
    } else {
#pragma unroll
        for (int q = 0; q < E::P; q++) x[q] = 0.0;
    }
}

// Children operands: grid (cols/128, rows, parents); the parent holds xr x
// xc elements (2 rows x 2 cols except where zero-extended).  A thread reads
// element (i, j) of the parent's four quadrants once and writes it to all
// seven children.  The sums are formed with add_int; a thread whose sums
// met a rare case forms them again with add and overwrites its children
// (the same thread's later stores win), so every child holds add's result.
template <class E, int SIDE>
__global__ void k_expand(int64_t rows, int64_t cols, int64_t xr, int64_t xc, View<const double> X, View<double> Y) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = blockIdx.y;
    int64_t p = blockIdx.z;
    if (j >= cols) return;
    constexpr int side = SIDE;
    double Q[4][E::P];
#pragma unroll
    for (int q = 0; q < 4; q++) ld_ext<E>(X, p, (q >> 1) * rows + i, (q & 1) * cols + j, xr, xc, Q[q]);
    bool rare = false;
#pragma unroll
    for (int c = 0; c < 7; c++) {
        const int qa = child_op(side, 0, c), qb = child_op(side, 1, c), op = child_op(side, 2, c);
        if (op == 0) {
            st<E>(Y, p * 7 + c, i, j, Q[qa]);
        } else {
            double y[E::P], r[E::P];
#pragma unroll
            for (int q = 0; q < E::P; q++) y[q] = op == 2 ? E::neg_int(Q[qb][q]) : Q[qb][q];
            E::add_int(Q[qa], y, r, rare);
            st<E>(Y, p * 7 + c, i, j, r);
        }
    }
    if (rare) {
#pragma unroll
        for (int c = 0; c < 7; c++) {
            const int qa = child_op(side, 0, c), qb = child_op(side, 1, c), op = child_op(side, 2, c);
            if (op != 0) {
                double y[E::P], r[E::P];
#pragma unroll
                for (int q = 0; q < E::P; q++) y[q] = op == 2 ? -Q[qb][q] : Q[qb][q];
                E::add(Q[qa], y, r);
                st<E>(Y, p * 7 + c, i, j, r);
            }
        }
    }
}

// The four quadrants of a parent element from its seven children (Eq 3):
// C11 = ((P1 + P4) - P5) + P7 and C22 = ((P1 + P3) - P2) + P6 advance side
// by side, C12 = P3 + P5 and C21 = P2 + P4 between them: four independent
// additions per step instead of one chain of eight (each result keeps its
// left-to-right order).  INT: add_int and neg_int (`rare` set where add is
// needed), else add.
template <class E, bool INT>
__device__ __forceinline__ void assemble(const double (&P)[7][E::P], double* c11, double* c12, double* c21,
                                         double* c22, bool& rare) {
    double n5[E::P], n2[E::P];
#pragma unroll
    for (int q = 0; q < E::P; q++) {
        n5[q] = INT ? E::neg_int(P[4][q]) : -P[4][q];
        n2[q] = INT ? E::neg_int(P[1][q]) : -P[1][q];
    }
    auto add = [&](const double* x, const double* y, double* z) {
        if (INT) E::add_int(x, y, z, rare);
        else E::add(x, y, z);
    };
    double a[E::P], b[E::P];
    add(P[0], P[3], a);
    add(P[0], P[2], b);
    add(P[2], P[4], c12);
    add(P[1], P[3], c21);
    double a2[E::P], b2[E::P];
    add(a, n5, a2);
    add(b, n2, b2);
    add(a2, P[6], c11);
    add(b2, P[5], c22);
}

// Parent products from children: grid (cols/128, rows, parents); only the
// first xr rows and xc columns of the parent are written.  The quadrants
// are assembled with add_int; a thread that met a rare case reads its
// children again, assembles with add and overwrites its outputs.
template <class E>
__global__ void k_combine(int64_t rows, int64_t cols, int64_t xr, int64_t xc, View<const double> Pc,
                          View<double> Out) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = blockIdx.y;
    int64_t p = blockIdx.z;
    if (j >= cols) return;
    double P[7][E::P];
#pragma unroll
    for (int c = 0; c < 7; c++) ld<E>(Pc, p * 7 + c, i, j, P[c]);
    double c11[E::P], c12[E::P], c21[E::P], c22[E::P];
    bool rare = false;
    assemble<E, true>(P, c11, c12, c21, c22, rare);
    const bool r0 = i < xr, r1 = rows + i < xr, c0 = j < xc, c1 = cols + j < xc;
    if (r0 && c0) st<E>(Out, p, i, j, c11);
    if (r0 && c1) st<E>(Out, p, i, cols + j, c12);
    if (r1 && c0) st<E>(Out, p, rows + i, j, c21);
    if (r1 && c1) st<E>(Out, p, rows + i, cols + j, c22);
    if (rare) {
#pragma unroll
        for (int c = 0; c < 7; c++) ld<E>(Pc, p * 7 + c, i, j, P[c]);
        assemble<E, false>(P, c11, c12, c21, c22, rare);
        if (r0 && c0) st<E>(Out, p, i, j, c11);
        if (r0 && c1) st<E>(Out, p, i, cols + j, c12);
        if (r1 && c0) st<E>(Out, p, rows + i, j, c21);
        if (r1 && c1) st<E>(Out, p, rows + i, cols + j, c22);
    }
}

// ---------------------------------------------------------------- multi-limb element ops

template <int W>
__device__ __forceinline__ void ldm(const View<const uint32_t>& V, int64_t z, int64_t i, int64_t j, MPV<W>& v) {
    const uint32_t* p = V.at(z, 0, i, j);
    v.e = (int)V.get(p);
    v.f = V.get(p + V.ps);
#pragma unroll
    for (int w = 0; w < W; w++) v.m[w] = V.get(p + (2 + w) * V.ps);
}
template <int W>
__device__ __forceinline__ void stm(const View<uint32_t>& V, int64_t z, int64_t i, int64_t j, const MPV<W>& v) {
    uint32_t* p = V.at(z, 0, i, j);
    V.store(p, (uint32_t)v.e);
    V.store(p + V.ps, v.f);
#pragma unroll
    for (int w = 0; w < W; w++) V.store(p + (2 + w) * V.ps, v.m[w]);
}

template <int W>
__device__ __forceinline__ void ldm_ext(const View<const uint32_t>& V, int64_t p, int64_t r, int64_t c, int64_t xr,
                                        int64_t xc, MPV<W>& v) {
    if (r < xr && c < xc) ldm<W>(V, p, r, c, v);
    else mp_set_zero(v, 0u);   // +0, the extension's value
}

template <int W>
__global__ void k_expand_mp(int64_t rows, int64_t cols, int64_t xr, int64_t xc, View<const uint32_t> X,
                            View<uint32_t> Y, ChildOps ops, unsigned* status) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = blockIdx.y;
    int z = blockIdx.z, p = z / 7, c = z % 7;
    if (j >= cols) return;
    int qa = ops.qa[c], qb = ops.qb[c], op = ops.op[c];
    MPV<W> x, y, r;
    ldm_ext<W>(X, p, (qa >> 1) * rows + i, (qa & 1) * cols + j, xr, xc, x);
    if (op == 0) {
        stm<W>(Y, z, i, j, x);
        return;
    }
    ldm_ext<W>(X, p, (qb >> 1) * rows + i, (qb & 1) * cols + j, xr, xc, y);
    if (op == 2) y.f ^= 1u;
    unsigned sts = 0u;
    mp_add<W>(x, y, r, sts);
    stm<W>(Y, z, i, j, r);
    if (sts) atomicOr(status, sts);
}

template <int W>
__global__ void k_combine_mp(int64_t rows, int64_t cols, int64_t xr, int64_t xc, View<const uint32_t> Pc,
                             View<uint32_t> Out, unsigned* status) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t i = blockIdx.y;
    int64_t p = blockIdx.z;
    if (j >= cols) return;
    const bool r0 = i < xr, r1 = rows + i < xr, c0 = j < xc, c1 = cols + j < xc;
    unsigned sts = 0u;
    MPV<W> a, b, t, u;
    // C11 = ((P1 + P4) - P5) + P7
    ldm<W>(Pc, p * 7 + 0, i, j, a);
    ldm<W>(Pc, p * 7 + 3, i, j, b);
    mp_add<W>(a, b, t, sts);
    ldm<W>(Pc, p * 7 + 4, i, j, b);
    b.f ^= 1u;
    mp_add<W>(t, b, u, sts);
    ldm<W>(Pc, p * 7 + 6, i, j, b);
    mp_add<W>(u, b, t, sts);
    if (r0 && c0) stm<W>(Out, p, i, j, t);
    // C12 = P3 + P5
    ldm<W>(Pc, p * 7 + 2, i, j, a);
    ldm<W>(Pc, p * 7 + 4, i, j, b);
    mp_add<W>(a, b, t, sts);
    if (r0 && c1) stm<W>(Out, p, i, cols + j, t);
    // C21 = P2 + P4
    ldm<W>(Pc, p * 7 + 1, i, j, a);
    ldm<W>(Pc, p * 7 + 3, i, j, b);
    mp_add<W>(a, b, t, sts);
    if (r1 && c0) stm<W>(Out, p, rows + i, j, t);
    // C22 = ((P1 + P3) - P2) + P6
    ldm<W>(Pc, p * 7 + 0, i, j, a);
    ldm<W>(Pc, p * 7 + 2, i, j, b);
    mp_add<W>(a, b, t, sts);
    ldm<W>(Pc, p * 7 + 1, i, j, b);
    b.f ^= 1u;
    mp_add<W>(t, b, u, sts);
    ldm<W>(Pc, p * 7 + 5, i, j, b);
    mp_add<W>(u, b, t, sts);
    if (r1 && c1) stm<W>(Out, p, rows + i, cols + j, t);
    if (sts) atomicOr(status, sts);
}

__global__ void k_fill_u32(uint32_t* p, size_t count, uint32_t v) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) p[i] = v;
}

int fill_u32(uint32_t* p, size_t count, uint32_t value, cudaStream_t s) {
    if (count == 0) return MPGEMM_OK;
    k_fill_u32<<<ceil_div((int64_t)count, 256), 256, 0, s>>>(p, count, value);
    return check_launch();
}

// ---------------------------------------------------------------- driver

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// x rounded up to a multiple of 2^depth (the zero-extended size).
int64_t strassen_extended(int64_t x, int depth) {
    const int64_t q = (int64_t)1 << depth;
    return (x + q - 1) / q * q;
}

size_t strassen_workspace_bytes(size_t eb, int64_t m, int64_t l, int64_t n, int depth) {
    m = strassen_extended(m, depth);
    l = strassen_extended(l, depth);
    n = strassen_extended(n, depth);
    size_t total = 0, nodes = 1;
    for (int k = 1; k <= depth; k++) {
        nodes *= 7;
        int64_t mk = m >> k, lk = l >> k, nk = n >> k;
        total += align256(nodes * (size_t)(mk * lk) * eb);
        total += align256(nodes * (size_t)(lk * nk) * eb);
        total += align256(nodes * (size_t)(mk * nk) * eb);
    }
    return total;
}

// Batched view of `count` contiguous r x c matrices with P planes each.
template <class T>
static View<T> batch_view(T* base, int64_t r, int64_t c, int P, size_t count) {
    View<T> v{base, c, r * c, (int64_t)P * r * c};
    return bounded(v, base, sizeof(T) * (size_t)P * (size_t)(r * c) * count);
}

template <class T>
struct Levels {
    View<T> SA[5], SB[5], PR[5];
};

template <class T>
static int carve(char* ws, size_t ws_bytes, size_t eb, int P, int64_t m, int64_t l, int64_t n, int depth,
                 Levels<T>& L) {
    size_t off = 0, nodes = 1;
    for (int k = 1; k <= depth; k++) {
        nodes *= 7;
        int64_t mk = m >> k, lk = l >> k, nk = n >> k;
        T* a = reinterpret_cast<T*>(ws + off);
        off += align256(nodes * (size_t)(mk * lk) * eb);
        T* b = reinterpret_cast<T*>(ws + off);
        off += align256(nodes * (size_t)(lk * nk) * eb);
        T* c = reinterpret_cast<T*>(ws + off);
        off += align256(nodes * (size_t)(mk * nk) * eb);
        L.SA[k] = batch_view(a, mk, lk, P, nodes);
        L.SB[k] = batch_view(b, lk, nk, P, nodes);
        L.PR[k] = batch_view(c, mk, nk, P, nodes);
    }
    return off <= ws_bytes ? MPGEMM_OK : MPGEMM_ENOMEM;
}

template <class T>
static View<const T> cview(const View<T>& v) {
    View<const T> r{v.p, v.ld, v.ps, v.bs};
#ifdef MPGEMM_BOUNDS_CHECK
    r.lo = v.lo;
    r.hi = v.hi;
    r.oob = v.oob;
#endif
    return r;
}

int strassen_ddqd_ws(int kind, int64_t m, int64_t l, int64_t n, View<const double> A, View<const double> B,
                     View<double> C, int n_min, int depth, void* ws, size_t ws_bytes, cudaStream_t s) {
    const int P = kind == MPGEMM_KIND_DD ? 2 : 4;
    const size_t eb = sizeof(double) * P;
    const int64_t mq = strassen_extended(m, depth), lq = strassen_extended(l, depth), nq = strassen_extended(n, depth);
    Levels<double> L;
    int rc = carve<double>((char*)ws, ws_bytes, eb, P, mq, lq, nq, depth, L);
    if (rc) return rc;
    unsigned parents = 1;
    for (int k = 1; k <= depth; k++) {
        int64_t mk = mq >> k, lk = lq >> k, nk = nq >> k;
        View<const double> pa = k == 1 ? A : cview(L.SA[k - 1]);
        View<const double> pb = k == 1 ? B : cview(L.SB[k - 1]);
        // level 1 reads the caller's m x l and l x n matrices, deeper levels whole parents
        const int64_t ar = k == 1 ? m : 2 * mk, ac = k == 1 ? l : 2 * lk, bc = k == 1 ? n : 2 * nk;
        dim3 ga(ceil_div(lk, 128), (unsigned)mk, parents), gb(ceil_div(nk, 128), (unsigned)lk, parents);
        if (kind == MPGEMM_KIND_DD) {
            k_expand<DDE, 0><<<ga, 128, 0, s>>>(mk, lk, ar, ac, pa, L.SA[k]);
            k_expand<DDE, 1><<<gb, 128, 0, s>>>(lk, nk, ac, bc, pb, L.SB[k]);
        } else {
            k_expand<QDE, 0><<<ga, 128, 0, s>>>(mk, lk, ar, ac, pa, L.SA[k]);
            k_expand<QDE, 1><<<gb, 128, 0, s>>>(lk, nk, ac, bc, pb, L.SB[k]);
        }
        if ((rc = check_launch())) return rc;
        parents *= 7;
    }
    rc = ddqd_gemm(kind, MPGEMM_BLOCK, mq >> depth, lq >> depth, nq >> depth, parents, cview(L.SA[depth]),
                   cview(L.SB[depth]), L.PR[depth], n_min, s);
    if (rc) return rc;
    for (int k = depth; k >= 1; k--) {
        parents /= 7;
        int64_t mk = mq >> k, nk = nq >> k;
        View<double> out = k == 1 ? C : L.PR[k - 1];
        const int64_t xr = k == 1 ? m : 2 * mk, xc = k == 1 ? n : 2 * nk;
        dim3 g(ceil_div(nk, 128), (unsigned)mk, parents);
        if (kind == MPGEMM_KIND_DD) k_combine<DDE><<<g, 128, 0, s>>>(mk, nk, xr, xc, cview(L.PR[k]), out);
        else k_combine<QDE><<<g, 128, 0, s>>>(mk, nk, xr, xc, cview(L.PR[k]), out);
        if ((rc = check_launch())) return rc;
    }
    return MPGEMM_OK;
}

template <int W>
static int strassen_mp_w(int64_t m, int64_t l, int64_t n, View<const uint32_t> A, View<const uint32_t> B,
                         View<uint32_t> C, int n_min, int depth, void* ws, size_t ws_bytes, cudaStream_t s) {
    const int P = 2 + W;
    const size_t eb = sizeof(uint32_t) * P;
    unsigned* status = device_status_ptr();
    if (!status) return MPGEMM_ECUDA;
    const int64_t mq = strassen_extended(m, depth), lq = strassen_extended(l, depth), nq = strassen_extended(n, depth);
    Levels<uint32_t> L;
    int rc = carve<uint32_t>((char*)ws, ws_bytes, eb, P, mq, lq, nq, depth, L);
    if (rc) return rc;
    const ChildOps ao = a_side_ops(), bo = b_side_ops();
    unsigned parents = 1;
    for (int k = 1; k <= depth; k++) {
        int64_t mk = mq >> k, lk = lq >> k, nk = nq >> k;
        View<const uint32_t> pa = k == 1 ? A : cview(L.SA[k - 1]);
        View<const uint32_t> pb = k == 1 ? B : cview(L.SB[k - 1]);
        const int64_t ar = k == 1 ? m : 2 * mk, ac = k == 1 ? l : 2 * lk, bc = k == 1 ? n : 2 * nk;
        dim3 ga(ceil_div(lk, 128), (unsigned)mk, parents * 7), gb(ceil_div(nk, 128), (unsigned)lk, parents * 7);
        k_expand_mp<W><<<ga, 128, 0, s>>>(mk, lk, ar, ac, pa, L.SA[k], ao, status);
        k_expand_mp<W><<<gb, 128, 0, s>>>(lk, nk, ac, bc, pb, L.SB[k], bo, status);
        if ((rc = check_launch())) return rc;
        parents *= 7;
    }
    rc = mp_gemm(W, MPGEMM_BLOCK, mq >> depth, lq >> depth, nq >> depth, parents, cview(L.SA[depth]),
                 cview(L.SB[depth]), L.PR[depth], n_min, s);
    if (rc) return rc;
    for (int k = depth; k >= 1; k--) {
        parents /= 7;
        int64_t mk = mq >> k, nk = nq >> k;
        View<uint32_t> out = k == 1 ? C : L.PR[k - 1];
        const int64_t xr = k == 1 ? m : 2 * mk, xc = k == 1 ? n : 2 * nk;
        dim3 g(ceil_div(nk, 128), (unsigned)mk, parents);
        k_combine_mp<W><<<g, 128, 0, s>>>(mk, nk, xr, xc, cview(L.PR[k]), out, status);
        if ((rc = check_launch())) return rc;
    }
    return MPGEMM_OK;
}

int strassen_mp_ws(int w, int64_t m, int64_t l, int64_t n, View<const uint32_t> A, View<const uint32_t> B,
                   View<uint32_t> C, int n_min, int depth, void* ws, size_t ws_bytes, cudaStream_t s) {
    switch (w) {
        case 1: return strassen_mp_w<1>(m, l, n, A, B, C, n_min, depth, ws, ws_bytes, s);
        case 2: return strassen_mp_w<2>(m, l, n, A, B, C, n_min, depth, ws, ws_bytes, s);
        case 4: return strassen_mp_w<4>(m, l, n, A, B, C, n_min, depth, ws, ws_bytes, s);
        case 8: return strassen_mp_w<8>(m, l, n, A, B, C, n_min, depth, ws, ws_bytes, s);
        case 16: return strassen_mp_w<16>(m, l, n, A, B, C, n_min, depth, ws, ws_bytes, s);
        case 32: return strassen_mp_w<32>(m, l, n, A, B, C, n_min, depth, ws, ws_bytes, s);
        case 64: return strassen_mp_w<64>(m, l, n, A, B, C, n_min, depth, ws, ws_bytes, s);
        default: return MPGEMM_EUNSUPPORTED;
    }
}

int strassen_ddqd(int kind, int64_t m, int64_t l, int64_t n, View<const double> A, View<const double> B,
                  View<double> C, int n_min, int depth, cudaStream_t s) {
    size_t bytes = strassen_workspace_bytes(sizeof(double) * (kind == MPGEMM_KIND_DD ? 2 : 4), m, l, n, depth);
    void* ws = nullptr;
    bool owned = false;
    int rc = workspace_get(bytes, s, &ws, &owned);
    if (rc) return rc;
    rc = strassen_ddqd_ws(kind, m, l, n, A, B, C, n_min, depth, ws, bytes, s);
    int rc2 = workspace_release(ws, owned, s);
    return rc ? rc : rc2;
}

int strassen_mp(int w, int64_t m, int64_t l, int64_t n, View<const uint32_t> A, View<const uint32_t> B,
                View<uint32_t> C, int n_min, int depth, cudaStream_t s) {
    size_t bytes = strassen_workspace_bytes(sizeof(uint32_t) * (size_t)(2 + w), m, l, n, depth);
    void* ws = nullptr;
    bool owned = false;
    int rc = workspace_get(bytes, s, &ws, &owned);
    if (rc) return rc;
    rc = strassen_mp_ws(w, m, l, n, A, B, C, n_min, depth, ws, bytes, s);
    int rc2 = workspace_release(ws, owned, s);
    return rc ? rc : rc2;
}

}  // namespace mpg
