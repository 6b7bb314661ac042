"""Pins of the oracle's split-precision (Ozaki-style) DD GEMM steps (no GPU).

* exponents: e_i is the largest frexp exponent of row i's hi words (and f_j
  of column j's), so every scaled |a'| < 1.
* slicing: sum_s d_s 2^(-7s) equals a' truncated toward zero to 7S bits,
  exactly (Fractions); every digit is an int8 in [-127, 127] with a's sign.
* level sums: equal to numpy int64 matrix products of the digit planes,
  summed over s + t = g (an independent library routine).
* recombination: equals the exact level sum rounded greedily to DD.
* end to end: |C - C_exact| <= 2^-100 |A||B| at S = 16 on row/column scaled
  inputs, and the error falls as S grows.
"""

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact import greedy, value
from paper_1710_01839_gb300 import inputs as I


def _frexp_exp(x: float) -> int:
    return math.frexp(x)[1]


def test_exponents_and_scaling():
    A, B = I.dd_rowcol_scaled(9, 13, 7, seed=3)
    e = oracle.ozaki_row_expo(A)
    f = oracle.ozaki_col_expo(B)
    for i in range(9):
        assert e[i] == max(_frexp_exp(x) for x in A[0, i] if x != 0)
        for k in range(13):
            assert abs(value(A[:, i, k])) < Fraction(2) ** int(e[i])
    for j in range(7):
        assert f[j] == max(_frexp_exp(x) for x in B[0, :, j] if x != 0)


def test_exponents_skip_zeros_of_small_rows():
    # rows and columns of magnitudes far below 1 with zeros among them: the
    # exponent is the largest over the nonzero entries (negative here), so a
    # zero must not count as exponent 0
    A, B = I.dd_rowcol_scaled(6, 8, 5, seed=11)
    A *= 2.0 ** -40
    B *= 2.0 ** -40
    A[:, :, 3] = 0.0
    B[:, 2, :] = 0.0
    e = oracle.ozaki_row_expo(A)
    f = oracle.ozaki_col_expo(B)
    for i in range(6):
        assert e[i] == max(_frexp_exp(x) for x in A[0, i] if x != 0) < 0
    for j in range(5):
        assert f[j] == max(_frexp_exp(x) for x in B[0, :, j] if x != 0) < 0


@pytest.mark.parametrize("S", [1, 3, 8, 16])
def test_digits_are_exact_truncation(S):
    A, _ = I.dd_rowcol_scaled(6, 10, 4, seed=4)
    A[:, 2, 3] = 0.0          # a zero element
    A[:, 4, :] = 0.0          # an all-zero row
    e = oracle.ozaki_row_expo(A)
    D = oracle.ozaki_slice(A, e, S, by_col=False)
    assert D.dtype == np.int8
    assert np.abs(D.astype(np.int64)).max() <= 127
    for i in range(6):
        for k in range(10):
            a = value(A[:, i, k]) * Fraction(2) ** -int(e[i])
            scaled = a * (1 << (7 * S))
            trunc = (abs(scaled.numerator) // scaled.denominator) * (1 if a >= 0 else -1)
            got = sum(int(D[s, i, k]) << (7 * (S - 1 - s)) for s in range(S))
            assert got == trunc
            if a > 0:
                assert (D[:, i, k] >= 0).all()
            if a < 0:
                assert (D[:, i, k] <= 0).all()


def test_level_sums_match_numpy_integer_products():
    S = 5
    A, B = I.dd_rowcol_scaled(7, 12, 5, seed=5)
    e, f = oracle.ozaki_row_expo(A), oracle.ozaki_col_expo(B)
    DA = oracle.ozaki_slice(A, e, S, by_col=False)
    DB = oracle.ozaki_slice(B, f, S, by_col=True)
    L = oracle.ozaki_levels(DA, DB, S)
    want = np.zeros_like(L)
    for s in range(1, S + 1):
        for t in range(1, S + 2 - s):
            want[s + t] += DA[s - 1].astype(np.int64) @ DB[t - 1].astype(np.int64)
    assert np.array_equal(L, want)


def test_recombination_is_exact_then_rounded():
    S = 6
    A, B = I.dd_rowcol_scaled(5, 8, 4, seed=6)
    e, f = oracle.ozaki_row_expo(A), oracle.ozaki_col_expo(B)
    DA = oracle.ozaki_slice(A, e, S, by_col=False)
    DB = oracle.ozaki_slice(B, f, S, by_col=True)
    L = oracle.ozaki_levels(DA, DB, S)
    C = oracle.ozaki_recombine(L, e, f, S)
    for i in range(5):
        for j in range(4):
            x = sum((Fraction(int(L[g, i, j])) * Fraction(2) ** (int(e[i]) + int(f[j]) - 7 * g)
                     for g in range(2, S + 2)), Fraction(0))
            assert C[:, i, j].tolist() == greedy(x, 2)
    assert np.array_equal(C, oracle.ozaki_gemm(A, B, S))


def _max_rel_err(A, B, C):
    m, n = C.shape[1], C.shape[2]
    ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    err, absab = oracle.exact_check(A, B, C, ii.ravel(), jj.ravel())
    return float(np.max(err / absab))


def test_end_to_end_error_bound_and_monotone_in_slices():
    A, B = I.dd_rowcol_scaled(24, 40, 20, seed=7)
    errs = {}
    for S in (8, 12, 14, 16, 18):
        errs[S] = _max_rel_err(A, B, oracle.ozaki_gemm(A, B, S))
    assert errs[16] <= 2.0**-100
    assert errs[18] <= errs[16] <= errs[14] <= errs[12] <= errs[8]
    assert errs[8] > 2.0**-100   # too few slices really does lose accuracy


@pytest.mark.slow
def test_error_curve_by_slices():
    # the split-precision workload's recipe at 64 x 512 x 64: each int8 slice
    # adds about 7 bits and each FP8 (base-32) slice about 5 until the final
    # DD rounding (about 2^-110 of |A||B| here) is all that is left; the
    # defaults S = 16 (int8) and S = 22 (FP8) are inside 2^-100
    import math
    A, B = I.dd_rowcol_scaled(64, 512, 64, seed=I.seed_for(3))
    lg = lambda C: math.log2(_max_rel_err(A, B, C))
    int8 = {S: lg(oracle.ozaki_gemm(A, B, S)) for S in range(12, 19)}
    fp8 = {S: lg(oracle.ozaki_gemm_b32(A, B, S)) for S in range(16, 25)}
    for curve, step, last in ((int8, 7, 15), (fp8, 5, 21)):
        keys = sorted(curve)
        assert all(curve[b] <= curve[a] + 1e-9 for a, b in zip(keys, keys[1:]))
        for S in keys:
            if S < last:
                assert abs((curve[S] - curve[S + 1]) - step) < 1.0, (S, curve)
        assert curve[keys[-1]] > -112
    assert int8[16] <= -100 and fp8[22] <= -100
    # the stress variant: A's columns and B's rows also scaled by 2^q_k,
    # q ~ U{-8..8}, so entries spread further below their row / column maxima
    A, B = I.dd_rowcol_scaled(64, 512, 64, seed=I.seed_for(3), inner_spread=8)
    assert lg(oracle.ozaki_gemm(A, B, 16)) <= -104 and lg(oracle.ozaki_gemm_b32(A, B, 22)) <= -104


def test_exact_on_integers():
    a = I.int_matrix(6, 9, 8, -100, 100)
    b = I.int_matrix(9, 5, 9, -100, 100)
    C = oracle.ozaki_gemm(I.ints_to_dd(a), I.ints_to_dd(b), 4)
    assert np.array_equal(C[0], (a @ b).astype(np.float64))
    assert not C[1].any()


# ---------------------------------------------------------------- balanced base-32 (FP8) digits

@pytest.mark.parametrize("S", [1, 4, 22, 24])
def test_b32_digits_are_exact_balanced_truncation(S):
    A, _ = I.dd_rowcol_scaled(6, 10, 4, seed=14)
    A[:, 2, 3] = 0.0
    A[:, 4, :] = 0.0
    e = oracle.ozaki_row_expo(A)
    D = oracle.ozaki_slice_b32(A, e, S, by_col=False)
    Di = D.astype(np.int64)
    assert np.abs(Di).max() <= 16                       # every digit exact in FP8 e4m3
    for i in range(6):
        for k in range(10):
            x = value(A[:, i, k]) * Fraction(2) ** -(int(e[i]) + 1)
            assert abs(x) < Fraction(1, 2)
            if x != 0:
                # lower digits of |x| lie in [-16, 15] (balanced), the top one in [0, 16]
                signed = Di[:, i, k] if x > 0 else -Di[:, i, k]
                assert signed[1:].max(initial=-16) <= 15 and 0 <= signed[0] <= 16
            scaled = x * (1 << (5 * S))
            trunc = (abs(scaled.numerator) // scaled.denominator) * (1 if x >= 0 else -1)
            got = sum(int(D[s, i, k]) * (32 ** (S - 1 - s)) for s in range(S))
            assert got == trunc


def test_b32_pipeline_recombination_and_bound():
    S = 22
    A, B = I.dd_rowcol_scaled(20, 36, 18, seed=15)
    e, f = oracle.ozaki_row_expo(A), oracle.ozaki_col_expo(B)
    DA = oracle.ozaki_slice_b32(A, e, S, False)
    DB = oracle.ozaki_slice_b32(B, f, S, True)
    L = oracle.ozaki_levels(DA, DB, S)
    want = np.zeros_like(L)
    for s in range(1, S + 1):
        for t in range(1, S + 2 - s):
            want[s + t] += DA[s - 1].astype(np.int64) @ DB[t - 1].astype(np.int64)
    assert np.array_equal(L, want)
    C = oracle.ozaki_recombine_bits(L, e, f, S, 5, 1)
    for i in (0, 7, 19):
        for j in (0, 17):
            x = sum((Fraction(int(L[g, i, j])) * Fraction(2) ** (int(e[i]) + int(f[j]) + 2 - 5 * g)
                     for g in range(2, S + 2)), Fraction(0))
            assert C[:, i, j].tolist() == greedy(x, 2)
    assert np.array_equal(C, oracle.ozaki_gemm_b32(A, B, S))
    errs = {s: _max_rel_err(A, B, oracle.ozaki_gemm_b32(A, B, s)) for s in (12, 18, 22)}
    assert errs[22] <= 2.0**-100 and errs[22] <= errs[18] <= errs[12]


# ---------------------------------------------------------------- expansions of T terms (QD)

def test_terms_digits_equal_dd_digits():
    """Two implementations of one definition: the exact-sum digit routine on
    DD inputs reproduces the DD digit routine (S exact base-32 steps)."""
    A, _ = I.dd_rowcol_scaled(9, 14, 4, seed=16)
    A[:, 2, :] = 0.0
    A[0, 3, 5] = 3.0                     # integer-valued entries with a small lo of either sign
    A[1, 3, 5] = -2.0**-60
    A[0, 3, 6] = -5.0
    A[1, 3, 6] = 2.0**-58
    e = oracle.ozaki_row_expo(A)
    for S in (1, 7, 22, 24):
        assert np.array_equal(oracle.ozaki_slice_b32_terms(A, e, S, by_col=False),
                              oracle.ozaki_slice_b32(A, e, S, by_col=False))
    f = oracle.ozaki_col_expo(A)
    assert np.array_equal(oracle.ozaki_slice_b32_terms(A, f, 22, by_col=True),
                          oracle.ozaki_slice_b32(A, f, 22, by_col=True))


@pytest.mark.parametrize("S", [1, 10, 48, 52])
def test_qd_digits_are_exact_balanced_truncation(S):
    A, _ = I.qd_rowcol_scaled(5, 9, 3, seed=17)
    A[:, 1, 4] = 0.0
    A[2:, 3, :] = 0.0                    # DD-like rows
    e = oracle.ozaki_row_expo(A)
    D = oracle.ozaki_slice_b32_terms(A, e, S, by_col=False)
    assert np.abs(D.astype(np.int64)).max() <= 16
    for i in range(5):
        for k in range(9):
            x = value(A[:, i, k]) * Fraction(2) ** -(int(e[i]) + 1)
            assert abs(x) < Fraction(1, 2)
            scaled = x * (1 << (5 * S))
            trunc = (abs(scaled.numerator) // scaled.denominator) * (1 if x >= 0 else -1)
            got = sum(int(D[s, i, k]) * (32 ** (S - 1 - s)) for s in range(S))
            assert got == trunc


def test_recombine_terms_two_equals_dd_recombination():
    S = 12
    A, B = I.dd_rowcol_scaled(7, 11, 6, seed=18)
    e, f = oracle.ozaki_row_expo(A), oracle.ozaki_col_expo(B)
    L = oracle.ozaki_levels(oracle.ozaki_slice_b32(A, e, S, False), oracle.ozaki_slice_b32(B, f, S, True), S)
    assert np.array_equal(oracle.ozaki_recombine_terms(L, e, f, S, 2), oracle.ozaki_recombine_bits(L, e, f, S, 5, 1))
    C4 = oracle.ozaki_recombine_terms(L, e, f, S, 4)
    for i in (0, 6):
        for j in (0, 5):
            x = sum((Fraction(int(L[g, i, j])) * Fraction(2) ** (int(e[i]) + int(f[j]) + 2 - 5 * g)
                     for g in range(2, S + 2)), Fraction(0))
            assert C4[:, i, j].tolist() == greedy(x, 4)
    assert np.array_equal(oracle.ozaki_gemm_b32_terms(A, B, 22), oracle.ozaki_gemm_b32(A, B, 22))


def test_qd_split_exact_on_integers_and_within_qd_bound():
    a, b = I.int_matrix(8, 12, 31, -1000, 1000), I.int_matrix(12, 7, 32, -1000, 1000)
    C = oracle.ozaki_gemm_b32_terms(I.ints_to_qd(a), I.ints_to_qd(b), 10)
    assert np.array_equal(C[0], (a @ b).astype(np.float64)) and not C[1:].any()
    m, l, n = 10, 16, 9
    A, B = I.qd_rowcol_scaled(m, l, n, seed=19, spread=4)
    C = oracle.ozaki_gemm_b32_terms(A, B, 48)
    errs = []
    for i in range(m):
        for j in range(n):
            ex = sum((value(A[:, i, k]) * value(B[:, k, j]) for k in range(l)), Fraction(0))
            absab = sum((abs(value(A[:, i, k]) * value(B[:, k, j])) for k in range(l)), Fraction(0))
            errs.append(abs(value(C[:, i, j]) - ex) / absab)
    # the QD tolerance 4 l 2^-208 |A||B|
    assert max(errs) <= 4 * l * Fraction(2) ** -208
