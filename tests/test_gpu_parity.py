"""Parity of the CUDA path (through the C ABI) with the oracle and with the
exact product.

Bars (written into each test):
  DD      |C - C_exact| <= 4 l 2^-104 |A||B| elementwise (and within twice
          that of the oracle, which meets the same bound)
  QD      |C - C_exact| <= 4 l 2^-208 |A||B|
  MP      bit-identical to the oracle (simple and block keep k ascending)
  Strassen on integer matrices: bit-identical to the simple algorithm
  DD Strassen: |C - C_exact| <= 2^-96 l max|A| max|B|
Sizes span several tiles with ragged tails; the bench's full-size launch
configurations are checked on sampled entries.
"""

import numpy as np
import pytest

import oracle
from gpu_util import DD_BOUND, QD_BOUND, bound_ratio, dev, host, sample_indices
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")


def _full(m, n):
    ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    return ii.ravel().astype(np.int64), jj.ravel().astype(np.int64)


# ---------------------------------------------------------------- DD

@pytest.mark.parametrize("algo,n_min", [("simple", 0), ("block", 16), ("block", 32), ("block", 64),
                                        ("block", 128), ("block", 256)])
def test_dd_ragged(algo, n_min):
    m, l, n = 131, 97, 77
    A, B = I.dd_random(m, l, 101, 20), I.dd_random(l, n, 102, 20)
    C = host(mpg.gemm_dd(dev(A), dev(B), algo=algo, n_min=n_min))
    ii, jj = _full(m, n)
    assert bound_ratio(A, B, C, ii, jj, DD_BOUND) <= 1.0
    Co = oracle.dd_gemm(A, B)
    err, absab = oracle.exact_check(A, B, Co, ii, jj)
    diff = np.abs((C[0] - Co[0]) + (C[1] - Co[1])).ravel()
    assert np.all(diff <= 2 * DD_BOUND * l * absab)


@pytest.mark.parametrize("algo", ["simple", "block"])
def test_dd_small_config_full(algo):
    # 128^3, hi ~ U[-1,1], lo = hi 2^-53 u: every entry against the exact product
    n = 128
    A, B = I.dd_random(n, n, I.seed_for(0)), I.dd_random(n, n, I.seed_for(0, 1))
    C = host(mpg.gemm_dd(dev(A), dev(B), algo=algo))
    ii, jj = _full(n, n)
    assert bound_ratio(A, B, C, ii, jj, DD_BOUND) <= 1.0


@pytest.mark.parametrize("n,n_min", [(1024, 32), (1024, 64), (2048, 64), (2048, 128)])
def test_dd_large_config_sampled(n, n_min):
    A = I.dd_random(n, n, I.seed_for(1), exp_spread=20)
    B = I.dd_random(n, n, I.seed_for(1, 1), exp_spread=20)
    C = host(mpg.gemm_dd(dev(A), dev(B), algo="block", n_min=n_min))
    ii, jj = sample_indices(n, n, 512, seed=n + n_min)
    assert bound_ratio(A, B, C, ii, jj, DD_BOUND) <= 1.0


def test_dd_worst_case_positive_inputs():
    # all terms positive: partial sums grow monotonically, the accumulator's
    # hardest case for the deferred renormalisation
    n = 512
    A, B = np.abs(I.dd_random(n, n, 7)), np.abs(I.dd_random(n, n, 8))
    A[1] = np.abs(A[1]) * 0.5
    C = host(mpg.gemm_dd(dev(A), dev(B), algo="block", n_min=64))
    ii, jj = sample_indices(n, n, 256, seed=3)
    assert bound_ratio(A, B, C, ii, jj, DD_BOUND) <= 1.0


# ---------------------------------------------------------------- QD

@pytest.mark.parametrize("algo,n_min", [("simple", 0), ("block", 16), ("block", 32), ("block", 128)])
def test_qd_ragged(algo, n_min):
    m, l, n = 67, 53, 45
    A, B = I.qd_random(m, l, 103, 20), I.qd_random(l, n, 104, 20)
    C = host(mpg.gemm_qd(dev(A), dev(B), algo=algo, n_min=n_min))
    ii, jj = _full(m, n)
    assert bound_ratio(A, B, C, ii, jj, QD_BOUND) <= 1.0


@pytest.mark.parametrize("n", [1024])
def test_qd_large_config_sampled(n):
    A = I.qd_random(n, n, I.seed_for(1, 2), exp_spread=20)
    B = I.qd_random(n, n, I.seed_for(1, 3), exp_spread=20)
    C = host(mpg.gemm_qd(dev(A), dev(B), algo="block", n_min=32))
    ii, jj = sample_indices(n, n, 256, seed=n)
    assert bound_ratio(A, B, C, ii, jj, QD_BOUND) <= 1.0


# ---------------------------------------------------------------- multi-limb

@pytest.mark.parametrize("w", [1, 2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("algo", ["simple", "block"])
def test_mp_ragged_bit_exact(w, algo):
    m, l, n = 37, 29, 23
    A, B = I.mp_random(m, l, w, 200 + w), I.mp_random(l, n, w, 300 + w)
    C = host(mpg.gemm_mp(dev(A), dev(B), 32 * w, algo=algo, n_min=32), mp=True)
    Co = oracle.mp_gemm(A, B, prec_bits=32 * w)
    assert np.array_equal(C, Co)
    assert mpg.stream_status() == 0


@pytest.mark.parametrize("w,n", [(4, 256), (8, 256), (16, 256), (32, 256), (64, 128), (4, 512)])
def test_mp_large_config_sampled_rows(w, n):
    A = I.mp_random(n, n, w, I.seed_for(2, w))
    B = I.mp_random(n, n, w, I.seed_for(2, 100 + w))
    C = host(mpg.gemm_mp(dev(A), dev(B), 32 * w, algo="block", n_min=16), mp=True)
    for r0 in (0, n // 2, n - 1):
        Co = oracle.mp_gemm(A, B, prec_bits=32 * w, rows=(r0, r0 + 1))
        assert np.array_equal(C[:, r0], Co[:, r0]), r0


def _set_mantissas(P, w, mask, values, rng):
    """Write mantissas (Python ints in [2^(p-1), 2^p)) drawn from `values`
    into the entries of the MP planes P where mask is set."""
    for r, c in zip(*np.nonzero(mask)):
        v = values[int(rng.integers(0, len(values)))]
        for q in range(w):
            P[2 + q, r, c] = (v >> (32 * q)) & 0xFFFFFFFF


@pytest.mark.parametrize("w", [4, 8, 16, 32, 64])
@pytest.mark.parametrize("algo", ["simple", "block"])
def test_mp_short_product_branches_bit_exact(w, algo):
    # the multiply's high-part product decides most roundings and leaves
    # ties and near-ties to the full product: structured limbs and
    # mantissas whose products are exact ties, near-ties and near the next
    # ulp reach both branches; bit-identical to the oracle
    p = 32 * w
    m, l, n = 19, 21, 17
    rng = np.random.default_rng(4100 + w)
    A, B = I.mp_structured(m, l, w, 4200 + w), I.mp_structured(l, n, w, 4300 + w)
    tie_makers = [(1 << (p - 1)) + 1, 3 << (p - 2), (1 << (p - 1)) + 3, (1 << p) - 1, 1 << (p - 1),
                  (1 << (p - 1)) + (1 << (p // 2))]
    _set_mantissas(A, w, rng.random((m, l)) < 0.5, tie_makers, rng)
    _set_mantissas(B, w, rng.random((l, n)) < 0.5, tie_makers, rng)
    C = host(mpg.gemm_mp(dev(A), dev(B), p, algo=algo, n_min=16), mp=True)
    assert np.array_equal(C, oracle.mp_gemm(A, B, prec_bits=p))
    assert mpg.stream_status() == 0


def _mp_planes(entries, w):
    """MP planes (2 + w, rows, cols) from a nested list of (sign, e, M)."""
    rows, cols = len(entries), len(entries[0])
    P = np.zeros((2 + w, rows, cols), dtype=np.uint32)
    for r in range(rows):
        for c in range(cols):
            sgn, e, M = entries[r][c]
            P[0, r, c] = np.int32(e).view(np.uint32)
            P[1, r, c] = sgn
            for q in range(w):
                P[2 + q, r, c] = (M >> (32 * q)) & 0xFFFFFFFF
    return P


@pytest.mark.parametrize("w", [1, 2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("algo", ["simple", "block"])
def test_mp_round_carry_out_bit_exact(w, algo):
    # roundings that carry out of the top limb (M all ones rounds up to
    # 2^p): in the multiply (a product just below 2^(2p-1) within half an
    # ulp) and in the add (1 - 2^-p plus just over half an ulp, plus an
    # exact tie with odd M); bit-identical to the oracle
    p = 32 * w
    x = (1 << (p - 1)) + 12345
    while True:    # y with x y in [2^(2p-1) - 2^(p-2), 2^(2p-1))
        y = ((1 << (2 * p - 1)) - 1) // x
        if 0 < (1 << (2 * p - 1)) - x * y <= (1 << (p - 2)) and y >= (1 << (p - 1)):
            break
        x += 1
    one = (0, 1, 1 << (p - 1))
    ones = (0, 0, (1 << p) - 1)                       # 1 - 2^-p
    over_half = (0, -p, (1 << (p - 1)) + 1)           # 2^(-p-1) + 2^(-2p)
    tie = (0, -p, 1 << (p - 1))                       # 2^(-p-1)
    zero = (0, 0, 0)
    A = _mp_planes([[(0, 0, x), zero], [ones, over_half], [ones, tie]], w)
    A[1, 0, 1] = 2                                    # the zero flag
    B = _mp_planes([[(0, 0, y), one], [one, one]], w)
    C = host(mpg.gemm_mp(dev(A), dev(B), p, algo=algo, n_min=16), mp=True)
    assert np.array_equal(C, oracle.mp_gemm(A, B, prec_bits=p))
    # x y rounds up to 1/2; 1 - 2^-p plus over half an ulp, and plus an
    # exact tie (odd M), round up to 1
    top = C[2 + w - 1].astype(np.int64)
    low = C[2:2 + w - 1].astype(np.int64)
    for (r, c), e in (((0, 0), 0), ((1, 1), 1), ((2, 1), 1)):
        assert C[0, r, c].view(np.int32) == e and top[r, c] == 0x80000000 and not low[:, r, c].any()
    assert mpg.stream_status() == 0


def test_mp_cancellation_and_zeros():
    # rows of A that are negatives of each other, zero entries, equal exponents
    w = 4
    m, l, n = 8, 16, 8
    A = I.mp_random(m, l, w, 400, emin=-2, emax=2)
    B = I.mp_random(l, n, w, 401, emin=-2, emax=2)
    A[:, 1] = A[:, 0]
    A[1, 1] ^= 1                       # row 1 = -row 0
    A[:, 2, 3] = 0
    A[1, 2, 3] = 2                     # a zero (M = 0, e = 0, zero flag)
    B[:, 5, :] = B[:, 4, :]
    B[1, 5, :] ^= 1                    # two rows of B cancel in every product sum
    C = host(mpg.gemm_mp(dev(A), dev(B), 128, algo="block"), mp=True)
    assert np.array_equal(C, oracle.mp_gemm(A, B, prec_bits=128))


# ---------------------------------------------------------------- Strassen

@pytest.mark.parametrize("depth", [1, 2, 3, 4])
@pytest.mark.parametrize("fmt", ["dd", "qd", "mp128"])
def test_strassen_integers_bit_exact(fmt, depth):
    m, l, n = 64, 48, 40
    a, b = I.int_matrix(m, l, 500 + depth), I.int_matrix(l, n, 600 + depth)
    if fmt == "dd":
        C = host(mpg.gemm_dd(dev(I.ints_to_dd(a)), dev(I.ints_to_dd(b)), algo="strassen", n_min=16, depth=depth))
        want = I.ints_to_dd(a @ b)
    elif fmt == "qd":
        C = host(mpg.gemm_qd(dev(I.ints_to_qd(a)), dev(I.ints_to_qd(b)), algo="strassen", n_min=16, depth=depth))
        want = I.ints_to_qd(a @ b)
    else:
        C = host(mpg.gemm_mp(dev(I.ints_to_mp(a, 4)), dev(I.ints_to_mp(b, 4)), 128, algo="strassen", n_min=16,
                             depth=depth), mp=True)
        want = I.ints_to_mp(a @ b, 4)
    assert np.array_equal(C, want)


@pytest.mark.parametrize("depth", [1, 2, 3, 4])
def test_dd_strassen_bound(depth):
    n = 256
    A, B = I.dd_random(n, n, 700), I.dd_random(n, n, 701)
    C = host(mpg.gemm_dd(dev(A), dev(B), algo="strassen", n_min=32, depth=depth))
    ii, jj = sample_indices(n, n, 400, seed=depth)
    err, _ = oracle.exact_check(A, B, C, ii, jj)
    amax = np.max(np.abs(A[0] + A[1]))
    bmax = np.max(np.abs(B[0] + B[1]))
    assert np.max(err) <= 2.0**-96 * n * amax * bmax


@pytest.mark.parametrize("depth", [1, 2])
def test_qd_strassen_bound(depth):
    n = 64
    A, B = I.qd_random(n, n, 702), I.qd_random(n, n, 703)
    C = host(mpg.gemm_qd(dev(A), dev(B), algo="strassen", n_min=16, depth=depth))
    ii, jj = _full(n, n)
    err, _ = oracle.exact_check(A, B, C, ii, jj)
    amax = np.max(np.abs(A[0]))
    bmax = np.max(np.abs(B[0]))
    assert np.max(err) <= 2.0**-200 * n * amax * bmax


@pytest.mark.parametrize("depth", [1, 2, 3, 4])
def test_mp_strassen_bit_exact_vs_oracle(depth):
    w, n = 4, 32
    A, B = I.mp_random(n, n, w, 710 + depth), I.mp_random(n, n, w, 720 + depth)
    C = host(mpg.gemm_mp(dev(A), dev(B), 128, algo="strassen", n_min=8, depth=depth), mp=True)
    Co = oracle.mp_gemm(A, B, prec_bits=128, algo="strassen", n_min=8, depth=depth)
    assert np.array_equal(C, Co)


# Sizes that 2^depth does not divide: A and B are zero-extended to the next
# multiple of 2^depth (the oracle makes the same reading), so integer
# products stay exact and the multi-limb result is the oracle's bit for bit.
@pytest.mark.parametrize("depth", [1, 2, 3, 4])
@pytest.mark.parametrize("fmt", ["dd", "qd", "mp128"])
def test_strassen_odd_sizes_integers_bit_exact(fmt, depth):
    m, l, n = 67, 45, 37
    a, b = I.int_matrix(m, l, 800 + depth), I.int_matrix(l, n, 810 + depth)
    if fmt == "dd":
        C = host(mpg.gemm_dd(dev(I.ints_to_dd(a)), dev(I.ints_to_dd(b)), algo="strassen", n_min=16, depth=depth))
        want = I.ints_to_dd(a @ b)
    elif fmt == "qd":
        C = host(mpg.gemm_qd(dev(I.ints_to_qd(a)), dev(I.ints_to_qd(b)), algo="strassen", n_min=16, depth=depth))
        want = I.ints_to_qd(a @ b)
    else:
        C = host(mpg.gemm_mp(dev(I.ints_to_mp(a, 4)), dev(I.ints_to_mp(b, 4)), 128, algo="strassen", n_min=16,
                             depth=depth), mp=True)
        want = I.ints_to_mp(a @ b, 4)
    assert np.array_equal(C, want)


@pytest.mark.parametrize("n,depth", [(255, 3), (257, 2), (1025, 3)])
def test_dd_strassen_odd_sizes_bound(n, depth):
    A, B = I.dd_random(n, n, 820 + depth), I.dd_random(n, n, 830 + depth)
    C = host(mpg.gemm_dd(dev(A), dev(B), algo="strassen", n_min=32, depth=depth))
    ii, jj = sample_indices(n, n, 300, seed=n)         # includes the last row and column
    err, _ = oracle.exact_check(A, B, C, ii, jj)
    amax = np.max(np.abs(A[0] + A[1]))
    bmax = np.max(np.abs(B[0] + B[1]))
    nq = -(-n // 2**depth) * 2**depth                   # the zero-extended inner dimension
    assert np.max(err) <= 2.0**-96 * nq * amax * bmax


@pytest.mark.parametrize("m,l,n,depth", [(33, 29, 31, 2), (5, 7, 3, 1), (17, 40, 9, 3)])
def test_mp_strassen_odd_sizes_bit_exact_vs_oracle(m, l, n, depth):
    A, B = I.mp_random(m, l, 4, 840 + depth), I.mp_random(l, n, 4, 850 + depth)
    C = host(mpg.gemm_mp(dev(A), dev(B), 128, algo="strassen", n_min=8, depth=depth), mp=True)
    Co = oracle.mp_gemm(A, B, prec_bits=128, algo="strassen", n_min=8, depth=depth)
    assert np.array_equal(C, Co)


@pytest.mark.parametrize("depth", [1, 2])
def test_mp2048_strassen_bit_exact_vs_oracle(depth):
    A, B = I.mp_random(20, 18, 64, 860 + depth), I.mp_random(18, 14, 64, 870 + depth)
    C = host(mpg.gemm_mp(dev(A), dev(B), 2048, algo="strassen", n_min=8, depth=depth), mp=True)
    Co = oracle.mp_gemm(A, B, prec_bits=2048, algo="strassen", n_min=8, depth=depth)
    assert np.array_equal(C, Co)


def test_strassen_with_caller_workspace():
    import torch
    n = 128
    A, B = I.dd_random(n, n, 730), I.dd_random(n, n, 731)
    ref = host(mpg.gemm_dd(dev(A), dev(B), algo="strassen", n_min=32, depth=2))
    ws = torch.empty(mpg.workspace_size("dd", n, n, n, algo="strassen", depth=2), dtype=torch.uint8, device="cuda")
    mpg.set_workspace(ws)
    try:
        got = host(mpg.gemm_dd(dev(A), dev(B), algo="strassen", n_min=32, depth=2))
        small = torch.empty(1024, dtype=torch.uint8, device="cuda")
        mpg.set_workspace(small)
        with pytest.raises(mpg.MpgemmError):
            mpg.gemm_dd(dev(A), dev(B), algo="strassen", n_min=32, depth=2)
    finally:
        mpg.set_workspace(None)
    assert np.array_equal(ref, got)


# ---------------------------------------------------------------- edge cases

def test_edge_cases_and_errors():
    import torch
    # empty inner dimension: C = 0
    A = dev(np.zeros((2, 5, 0)))
    B = dev(np.zeros((2, 0, 4)))
    C = host(mpg.gemm_dd(A, B))
    assert C.shape == (2, 5, 4) and not C.any()
    Am = dev(np.zeros((6, 3, 0), dtype=np.uint32))
    Bm = dev(np.zeros((6, 0, 2), dtype=np.uint32))
    Cm = host(mpg.gemm_mp(Am, Bm, 128), mp=True)
    assert (Cm[1] == 2).all() and not Cm[0].any() and not Cm[2:].any()
    # empty output
    C = mpg.gemm_dd(dev(np.zeros((2, 0, 3))), dev(np.zeros((2, 3, 4))))
    assert C.shape == (2, 0, 4)
    # 1 x 1 x 1
    a = np.array([[[0.5]], [[2.0**-60]]])
    b = np.array([[[3.0]], [[0.0]]])
    c = host(mpg.gemm_dd(dev(a), dev(b), algo="simple"))
    assert c[0, 0, 0] + c[1, 0, 0] == 1.5 + 3 * 2.0**-60 and c[0, 0, 0] == 1.5
    # argument errors come back as status codes, nothing launched
    Ad, Bd = dev(I.dd_random(8, 8, 1)), dev(I.dd_random(8, 8, 2))
    with pytest.raises(mpg.MpgemmError) as e:
        mpg.gemm_dd(Ad, Bd, n_min=48)
    assert e.value.status == -1
    with pytest.raises(mpg.MpgemmError) as e:
        mpg.gemm_dd(Ad, Bd, C=Ad)               # C overlaps A
    assert e.value.status == -1
    L = mpg.lib()
    assert L.mpgemm_dd(-1, 1, 1, None, None, None, 1, 0, 0, None) == -1
    assert L.mpgemm_mp(2, 2, 2, 96, None, None, None, 1, 0, 0, None) == -2
    assert mpg.stream_status() == 0


def test_paper_matrices_dd_closed_form():
    # Section 4's matrices: c_ij = sqrt(15) n(n-1)(3i+n-2)/6 for every j
    n = 256
    A, B = I.paper_matrices(n, "dd")
    C = host(mpg.gemm_dd(dev(A), dev(B), algo="block", n_min=64))
    from fractions import Fraction
    import math
    r15 = Fraction(math.isqrt(15 << 600), 1 << 300)
    for i in (1, 2, n // 2, n):
        truth = r15 * I.paper_closed_form(n, i)
        for j in (0, n // 3, n - 1):
            got = Fraction(C[0, i - 1, j]) + Fraction(C[1, i - 1, j])
            assert abs(got - truth) <= (4 * n + 3) * Fraction(2) ** -104 * truth


# ---------------------------------------------------------------- the bench's own launch configurations

@pytest.mark.parametrize("depth", [3, 4])
def test_dd_bench_configuration_sampled(depth):
    """DD 2048^3 with the bench's inputs and its tuned launch (Strassen depth
    4, n_min 32; depth 3 the earlier choice): sampled entries against the
    exact product, Strassen bound."""
    n = 2048
    A = I.dd_random(n, n, I.seed_for(1, 0), exp_spread=20)
    B = I.dd_random(n, n, I.seed_for(1, 1), exp_spread=20)
    C = host(mpg.gemm_dd(dev(A), dev(B), algo="strassen", n_min=32, depth=depth))
    ii, jj = sample_indices(n, n, 384, seed=2048)
    err, _ = oracle.exact_check(A, B, C, ii, jj)
    amax, bmax = np.max(np.abs(A[0] + A[1])), np.max(np.abs(B[0] + B[1]))
    assert np.max(err) <= 2.0**-96 * n * amax * bmax


@pytest.mark.parametrize("depth", [3, 4])
def test_qd_bench_configuration_sampled(depth):
    n = 1024
    A = I.qd_random(n, n, I.seed_for(1, 0), exp_spread=20)
    B = I.qd_random(n, n, I.seed_for(1, 1), exp_spread=20)
    C = host(mpg.gemm_qd(dev(A), dev(B), algo="strassen", n_min=16, depth=depth))
    ii, jj = sample_indices(n, n, 128, seed=1024)
    err, _ = oracle.exact_check(A, B, C, ii, jj)
    assert np.max(err) <= 2.0**-200 * n * np.max(np.abs(A[0])) * np.max(np.abs(B[0]))


def test_mp256_bench_configuration_sampled():
    """256-bit 1024^3 with the bench's inputs and tuned launch (Strassen
    depth 3, n_min 512): sampled entries exactly (Fractions) within
    2^-(p-8) l max|A| max|B|, the multi-limb Strassen tolerance."""
    from fractions import Fraction
    from exact import mp_words_to_fraction
    n, w = 1024, 8
    A = I.mp_random(n, n, w, I.seed_for(2, w))
    B = I.mp_random(n, n, w, I.seed_for(2, w + 1))
    C = host(mpg.gemm_mp(dev(A), dev(B), 256, algo="strassen", n_min=512, depth=3), mp=True)
    fa = lambda X, i, k: mp_words_to_fraction(X[:, i, k], w)
    # max|A| max|B| < 2^64 2^64: exponents are at most 64 and mantissas below 1
    tol = Fraction(2) ** -(256 - 8) * n * Fraction(2) ** 128
    rng = np.random.default_rng(5)
    for _ in range(12):
        i, j = int(rng.integers(0, n)), int(rng.integers(0, n))
        ex = sum((fa(A, i, k) * fa(B, k, j) for k in range(n)), Fraction(0))
        assert abs(mp_words_to_fraction(C[:, i, j], w) - ex) <= tol


@pytest.mark.parametrize("w", [1, 4, 8, 64])
@pytest.mark.parametrize("algo", ["simple", "block"])
def test_mp_exponent_range_is_flagged(w, algo):
    # exponents are int32: a product past 2^31 - 1 (or below -2^31), and a
    # sum whose rounding carries the exponent of 2^31 - 1 one further, set
    # MPGEMM_EOVERFLOW; in-range neighbours of the same calls do not
    p = 32 * w
    top = 2 ** 31 - 1
    one = (0, 1, 1 << (p - 1))
    cases = {
        "mul_over": ([[(0, top - 5, 1 << (p - 1))]], [[(0, 10, 1 << (p - 1))]]),
        "mul_under": ([[(1, -2 ** 31 + 5, 1 << (p - 1))]], [[(0, -10, 1 << (p - 1))]]),
        "add_carry": ([[(0, top, (1 << p) - 1), (0, top - p, (1 << (p - 1)) + 1)]], [[one], [one]]),
        "in_range": ([[(0, top - 20, 1 << (p - 1))]], [[(0, 10, 1 << (p - 1))]]),
    }
    for name, (a, b) in cases.items():
        A, B = _mp_planes(a, w), _mp_planes(b, w)
        mpg.gemm_mp(dev(A), dev(B), p, algo=algo, n_min=16)
        want = 0 if name == "in_range" else -4
        assert mpg.stream_status() == want, name


# ---------------------------------------------------------------- measured margins at the bench's sizes

def test_strassen_error_margins_at_bench_sizes(capsys):
    # the bench's DD 2048^3 and QD 1024^3 inputs (exponent spread 2^[-20, 20]);
    # normwise |C - AB| / (l max|A| max|B|) against the Strassen bounds
    # (2^-96 DD, 2^-200 QD) and elementwise |C - AB| / |A||B| for the block
    # algorithm, on 512 random entries, row 0, column 0 and the corners
    import math
    rows = []
    for fmt, n, f, bound, cases in (
            ("dd", 2048, mpg.gemm_dd, 2.0**-96, [("block", 32, 0), ("strassen", 32, 1), ("strassen", 32, 2),
                                                   ("strassen", 32, 3), ("strassen", 32, 4)]),
            ("qd", 1024, mpg.gemm_qd, 2.0**-200, [("block", 16, 0), ("strassen", 16, 3), ("strassen", 16, 4)])):
        gen = I.dd_random if fmt == "dd" else I.qd_random
        A, B = gen(n, n, I.seed_for(1, 0), exp_spread=20), gen(n, n, I.seed_for(1, 1), exp_spread=20)
        Ad, Bd = dev(A), dev(B)
        ii, jj = sample_indices(n, n, 512, seed=5)
        scale = n * float(np.max(np.abs(A[0]))) * float(np.max(np.abs(B[0])))
        for algo, nm, d in cases:
            err, absab = oracle.exact_check(A, B, host(f(Ad, Bd, algo=algo, n_min=nm, depth=d)), ii, jj)
            norm, elem = float(np.max(err)) / scale, float(np.max(err / absab))
            assert norm <= bound
            if algo == "block":
                assert elem <= (DD_BOUND if fmt == "dd" else QD_BOUND) * n
            rows.append(f"{fmt} {n}^3 {algo} d={d}: normwise 2^{math.log2(max(norm, 1e-300)):.1f}, "
                        f"elementwise 2^{math.log2(max(elem, 1e-300)):.1f}")
    with capsys.disabled():
        print("\n" + "\n".join(rows))
