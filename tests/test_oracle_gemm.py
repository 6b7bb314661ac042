"""Pins of the oracle's GEMM algorithms (Eqs 1-3) without a GPU.

* Eq 2 (block, in-place accumulation over K blocks) is bit-identical to
  Eq 1 (simple) for every format, ragged sizes included.
* Eq 3 (Strassen) is bit-identical to Eq 1 on small integer matrices, where
  every intermediate is exact, at depths 1-4 in every format.
* DD and QD results lie within 4 l 2^-104 |A||B| (DD) and 4 l 2^-208 |A||B|
  (QD) of the exact product, computed with Fractions; DD Strassen within
  2^-96 l max|A| max|B|.
* The oracle's exact checker (used on large sampled problems) agrees with
  Fractions.
* Multi-limb GEMM is bit-identical to the same multiply/add sequence run
  with mpmath's correctly rounded operations.
* The paper's matrices (Section 4) reproduce the closed form
  c_ij = sqrt(15) n(n-1)(3i+n-2)/6 within the formats' bounds.
"""

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact import F, mp_words_to_fraction, value
from paper_1710_01839_gb300 import inputs as I


def _exact_product(A, B):
    T, m, l = A.shape
    n = B.shape[2]
    Af = [[sum(F(A[t, i, k]) for t in range(T)) for k in range(l)] for i in range(m)]
    Bf = [[sum(F(B[t, k, j]) for t in range(T)) for j in range(n)] for k in range(l)]
    C = [[sum((Af[i][k] * Bf[k][j] for k in range(l)), Fraction(0)) for j in range(n)] for i in range(m)]
    absab = [[sum((abs(Af[i][k]) * abs(Bf[k][j]) for k in range(l)), Fraction(0)) for j in range(n)] for i in range(m)]
    return C, absab


# ---------------------------------------------------------------- block == simple

@pytest.mark.parametrize("fmt", ["dd", "qd", "mp128", "mp256"])
def test_block_equals_simple_ragged(fmt):
    m, l, n = 13, 17, 11
    if fmt == "dd":
        A, B = I.dd_random(m, l, 11, 5), I.dd_random(l, n, 12, 5)
        run = oracle.dd_gemm
        kw = {}
    elif fmt == "qd":
        A, B = I.qd_random(m, l, 13, 5), I.qd_random(l, n, 14, 5)
        run = oracle.qd_gemm
        kw = {}
    else:
        p = int(fmt[2:])
        A, B = I.mp_random(m, l, p // 32, 15), I.mp_random(l, n, p // 32, 16)
        run = oracle.mp_gemm
        kw = {"prec_bits": p}
    C0 = run(A, B, algo="simple", **kw)
    for n_min in (1, 4, 5, 16, 64):
        C1 = run(A, B, algo="block", n_min=n_min, **kw)
        assert np.array_equal(C0, C1), n_min
    # a row range of the block algorithm equals the same rows of the full result
    C2 = run(A, B, algo="block", n_min=4, rows=(3, 9), **kw)
    assert np.array_equal(C2[:, 3:9], C0[:, 3:9])


# ---------------------------------------------------------------- Strassen == simple on integers

@pytest.mark.parametrize("depth", [1, 2, 3, 4])
@pytest.mark.parametrize("fmt", ["dd", "qd", "mp128"])
def test_strassen_equals_simple_on_integers(fmt, depth):
    m, l, n = 16, 24, 8
    a = I.int_matrix(m, l, 20 + depth)
    b = I.int_matrix(l, n, 30 + depth)
    exact = a @ b
    if fmt == "dd":
        A, B, run, kw = I.ints_to_dd(a), I.ints_to_dd(b), oracle.dd_gemm, {}
        want = I.ints_to_dd(exact)
    elif fmt == "qd":
        A, B, run, kw = I.ints_to_qd(a), I.ints_to_qd(b), oracle.qd_gemm, {}
        want = I.ints_to_qd(exact)
    else:
        A, B, run, kw = I.ints_to_mp(a, 4), I.ints_to_mp(b, 4), oracle.mp_gemm, {"prec_bits": 128}
        want = I.ints_to_mp(exact, 4)
    Cs = run(A, B, algo="simple", **kw)
    Ct = run(A, B, algo="strassen", n_min=2, depth=depth, **kw)
    assert np.array_equal(Cs, Ct)
    assert np.array_equal(Cs, want)


# Dimensions that 2^depth does not divide run on zero-extended matrices: on
# integer matrices every intermediate is still exact, so the result is the
# exact product, bit-identical to Eq 1, at any depth.
@pytest.mark.parametrize("depth", [1, 2, 3, 4])
@pytest.mark.parametrize("fmt", ["dd", "qd", "mp128"])
@pytest.mark.parametrize("m,l,n", [(13, 21, 7), (1, 5, 3), (9, 8, 17)])
def test_strassen_odd_dimensions_equal_simple_on_integers(fmt, depth, m, l, n):
    a = I.int_matrix(m, l, 40 + depth)
    b = I.int_matrix(l, n, 50 + depth)
    if fmt == "dd":
        A, B, run, kw, want = I.ints_to_dd(a), I.ints_to_dd(b), oracle.dd_gemm, {}, I.ints_to_dd(a @ b)
    elif fmt == "qd":
        A, B, run, kw, want = I.ints_to_qd(a), I.ints_to_qd(b), oracle.qd_gemm, {}, I.ints_to_qd(a @ b)
    else:
        A, B, run, kw = I.ints_to_mp(a, 4), I.ints_to_mp(b, 4), oracle.mp_gemm, {"prec_bits": 128}
        want = I.ints_to_mp(a @ b, 4)
    Ct = run(A, B, algo="strassen", n_min=2, depth=depth, **kw)
    assert np.array_equal(Ct, want)
    assert np.array_equal(Ct, run(A, B, algo="simple", **kw))


def test_dd_strassen_odd_dimensions_within_bound_of_exact():
    m, l, n = 11, 19, 13
    A, B = I.dd_random(m, l, 61, 20), I.dd_random(l, n, 62, 20)
    C = oracle.dd_gemm(A, B, algo="strassen", n_min=2, depth=2)
    Cx, _ = _exact_product(A, B)
    amax = max(abs(value(A[:, i, k])) for i in range(m) for k in range(l))
    bmax = max(abs(value(B[:, k, j])) for k in range(l) for j in range(n))
    tol = Fraction(2) ** -96 * 20 * amax * bmax   # 20: the zero-extended inner dimension
    for i in range(m):
        for j in range(n):
            assert abs(value(C[:, i, j]) - Cx[i][j]) <= tol


# ---------------------------------------------------------------- error bounds vs exact

def test_dd_simple_within_bound_of_exact():
    m, l, n = 6, 37, 5
    A, B = I.dd_random(m, l, 41, 20), I.dd_random(l, n, 42, 20)
    C = oracle.dd_gemm(A, B)
    Cx, absab = _exact_product(A, B)
    worst = 0.0
    for i in range(m):
        for j in range(n):
            err = abs(value(C[:, i, j]) - Cx[i][j])
            bound = 4 * l * Fraction(2) ** -104 * absab[i][j]
            assert err <= bound
            worst = max(worst, float(err / bound))
    assert worst > 0   # the oracle rounds: a zero error everywhere would mean the check is vacuous


def test_qd_simple_within_bound_of_exact():
    m, l, n = 4, 19, 3
    A, B = I.qd_random(m, l, 43, 20), I.qd_random(l, n, 44, 20)
    C = oracle.qd_gemm(A, B)
    Cx, absab = _exact_product(A, B)
    for i in range(m):
        for j in range(n):
            err = abs(value(C[:, i, j]) - Cx[i][j])
            assert err <= 4 * l * Fraction(2) ** -208 * absab[i][j]


def test_dd_strassen_within_bound_of_exact():
    n = 32
    A, B = I.dd_random(n, n, 45), I.dd_random(n, n, 46)
    C = oracle.dd_gemm(A, B, algo="strassen", n_min=4, depth=3)
    Cx, _ = _exact_product(A, B)
    amax = max(abs(value(A[:, i, k])) for i in range(n) for k in range(n))
    bmax = max(abs(value(B[:, i, k])) for i in range(n) for k in range(n))
    tol = Fraction(2) ** -96 * n * amax * bmax
    for i in range(n):
        for j in range(n):
            assert abs(value(C[:, i, j]) - Cx[i][j]) <= tol


@pytest.mark.parametrize("terms", [2, 4])
def test_exact_checker_matches_fractions(terms):
    m, l, n = 5, 11, 4
    gen = I.dd_random if terms == 2 else I.qd_random
    A, B = gen(m, l, 47, 10), gen(l, n, 48, 10)
    C = oracle.dd_gemm(A, B) if terms == 2 else oracle.qd_gemm(A, B)
    ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    err, absab = oracle.exact_check(A, B, C, ii.ravel(), jj.ravel())
    Cx, Ax = _exact_product(A, B)
    ent = oracle.exact_entries(A, B, ii.ravel(), jj.ravel(), terms)
    for s, (i, j) in enumerate(zip(ii.ravel(), jj.ravel())):
        assert err[s] == float(abs(Cx[i][j] - value(C[:, i, j])))
        assert absab[s] == float(Ax[i][j])
        x = Cx[i][j]
        for t in range(terms):
            assert ent[s, t] == float(x)
            x -= F(ent[s, t])


# ---------------------------------------------------------------- multi-limb sequence vs mpmath

@pytest.mark.parametrize("w", [2, 4])
def test_mp_gemm_matches_mpmath_sequence(w):
    mpm = pytest.importorskip("mpmath")
    from mpmath.libmp import fzero, from_man_exp, mpf_add, mpf_mul
    p = 32 * w
    m, l, n = 4, 9, 3
    A, B = I.mp_random(m, l, w, 50 + w), I.mp_random(l, n, w, 60 + w)
    C = oracle.mp_gemm(A, B, prec_bits=p)

    def to_mpf(words):
        v = mp_words_to_fraction(words, w)
        if v == 0:
            return fzero
        e = np.uint32(words[0]).view(np.int32).item()
        M = sum(int(words[2 + i]) << (32 * i) for i in range(w))
        return from_man_exp(-M if words[1] & 1 else M, e - p)

    for i in range(m):
        for j in range(n):
            c = fzero
            for k in range(l):
                t = mpf_mul(to_mpf(A[:, i, k]), to_mpf(B[:, k, j]), p, "n")
                c = mpf_add(c, t, p, "n")
            sign, man, exp, bc = c
            got = mp_words_to_fraction(C[:, i, j], w)
            want = Fraction(-man if sign else man) * Fraction(2) ** exp
            assert got == want


@pytest.mark.parametrize("algo", ["simple", "block"])
def test_mp_gemm_zero_signs_follow_ieee_rules(algo):
    # IEEE 754 round-to-nearest: an exact zero sum of opposite-signed operands
    # is +0, (-0) + (-0) = -0, and a product's sign is the XOR of its
    # operands'.  Eq 1's sum starts from the empty sum, +0, so an entry whose
    # products are all zeros is +0 whatever their signs.  (Eq 3 is left out:
    # its rounded sums of P1..P7 need not cancel to zero on a zero row.)
    w, m, l, n = 2, 4, 6, 4
    A, B = I.mp_random(m, l, w, 91), I.mp_random(l, n, w, 92)
    A[:, 1, :] = 0
    A[1, 1, :] = 3                       # row 1 of A: all -0
    B[:, :, 2] = 0
    B[1, :, 2] = 2                       # column 2 of B: all +0
    C = oracle.mp_gemm(A, B, prec_bits=32 * w, algo=algo, n_min=2)
    for i in range(m):
        for j in range(n):
            if i == 1 or j == 2:
                assert int(C[1, i, j]) == 2, (i, j, int(C[1, i, j]))    # +0
            else:
                assert int(C[1, i, j]) & 2 == 0


# ---------------------------------------------------------------- the paper's matrices

def _sqrt15_times(q: Fraction, bits=400) -> Fraction:
    # sqrt(15) * q, q >= 0, to within 2^-bits relative (plenty for the bounds below)
    r = Fraction(math.isqrt(15 << (2 * bits)), 1 << bits)
    return r * q


@pytest.mark.parametrize("fmt", ["dd", "qd", "mp128", "mp256"])
def test_paper_matrices_closed_form(fmt):
    n = 24
    if fmt in ("dd", "qd"):
        A, B = I.paper_matrices(n, fmt)
        C = oracle.dd_gemm(A, B, algo="block", n_min=8) if fmt == "dd" else oracle.qd_gemm(A, B, algo="block", n_min=8)
        rel = (4 * n + 3) * (Fraction(2) ** -104 if fmt == "dd" else Fraction(2) ** -208)
        get = lambda i, j: value(C[:, i, j])
    else:
        p = int(fmt[2:])
        w = p // 32
        A, B = I.paper_matrices(n, "mp", w)
        C = oracle.mp_gemm(A, B, prec_bits=p, algo="block", n_min=8)
        rel = (n + 3) * Fraction(2) ** (1 - p)
        get = lambda i, j: mp_words_to_fraction(C[:, i, j], w)
    for i in range(1, n + 1):
        truth = _sqrt15_times(I.paper_closed_form(n, i))
        for j in (1, n // 2, n):
            c = get(i - 1, j - 1)
            assert abs(c - truth) <= rel * truth, (i, j)
    # every column of a row is the same closed-form value up to rounding
    assert truth > 0
