"""The seeded input generators follow their stated recipes (no GPU).

Shapes and dtypes of the ABI layouts; the same seed gives the same matrix
and another seed another; DD / QD expansions are canonical (each term at
most half an ulp of the one before, re-represented without changing the
value); exponent spreads, scalings and value sets as documented; the integer
and closed-form matrices hold exactly the values they name."""

import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1710_01839_gb300 import inputs as I


def _half_ulp_ok(hi, lo):
    mag = np.abs(hi)
    up = np.nextafter(mag, np.inf) - mag
    dn = mag - np.nextafter(mag, 0.0)
    along = lo * np.sign(hi)
    # |lo| <= ulp(hi) / 2, measured toward the neighbour on lo's side
    return bool(np.all((mag == 0) & (lo == 0) | (along <= up / 2) & (-along <= dn / 2)))


def _mp_value(Y, w, idx):
    e = int(Y[0].reshape(-1).view(np.int32)[idx])
    f = int(Y[1].reshape(-1)[idx])
    if f & 2:
        return Fraction(0)
    M = sum(int(Y[2 + q].reshape(-1)[idx]) << (32 * q) for q in range(w))
    v = Fraction(M) * Fraction(2) ** (e - 32 * w)
    return -v if f & 1 else v


def test_dd_random_recipe():
    X = I.dd_random(40, 50, 1)
    assert X.shape == (2, 40, 50) and X.dtype == np.float64 and X.flags["C_CONTIGUOUS"]
    assert np.array_equal(X, I.dd_random(40, 50, 1)) and not np.array_equal(X, I.dd_random(40, 50, 2))
    assert np.all(np.abs(X[0]) <= 1.0) and _half_ulp_ok(X[0], X[1])
    # lo is a genuine second word (about 2^-53 |hi|), not zero
    assert np.mean(X[1] != 0) > 0.99
    assert np.all(np.abs(X[1]) <= np.abs(X[0]) * 2.0 ** -52)
    # the exponent spread multiplies both words by 2^k, k ~ U{-20..20}
    Y = I.dd_random(200, 200, 1, exp_spread=20)
    assert _half_ulp_ok(Y[0], Y[1])
    e = np.frexp(Y[0][Y[0] != 0])[1]
    assert e.max() - e.min() >= 40


def test_qd_random_recipe():
    X = I.qd_random(30, 30, 3, exp_spread=20)
    assert X.shape == (4, 30, 30)
    assert np.array_equal(X, I.qd_random(30, 30, 3, exp_spread=20))
    for t in range(3):
        assert _half_ulp_ok(X[t], X[t + 1])
    assert np.mean(X[3] != 0) > 0.99


@pytest.mark.parametrize("gen", [I.mp_random, I.mp_structured])
@pytest.mark.parametrize("w", [1, 4, 8, 64])
def test_mp_generators_are_normalised(gen, w):
    Y = gen(12, 9, w, 5)
    assert Y.shape == (2 + w, 12, 9) and Y.dtype == np.uint32
    assert np.array_equal(Y, gen(12, 9, w, 5))
    assert np.all(Y[2 + w - 1] >> 31 == 1)                 # top bit of the top limb
    assert set(np.unique(Y[1]).tolist()) <= {0, 1}         # signs, no zero flags
    e = Y[0].view(np.int32)
    lo, hi = (-64, 64) if gen is I.mp_random else (-8, 8)
    assert e.min() >= lo and e.max() <= hi


def test_mp_structured_value_set():
    Y = I.mp_structured(40, 40, 8, 6)
    special = {0, 1, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF}
    limbs = Y[2:2 + 7].reshape(-1).tolist()
    share = sum(v in special for v in limbs) / len(limbs)
    assert 0.75 < share < 0.9                               # 5 of 6 picks are special


def test_canonical_rewrite_keeps_the_value():
    # overlapping terms (each only 2^-20 below the one before), zeros between
    # them and cancelling neighbours: the rewrite is exact and canonical
    rng = np.random.default_rng(12)
    x = np.empty((4, 300))
    x[0] = rng.uniform(-1, 1, 300)
    for t in range(3):
        x[t + 1] = x[t] * 2.0 ** -20 * rng.uniform(-1, 1, 300)
    x[1, :20] = 0.0
    x[2, 20:40] = -x[1, 20:40]
    y = I._canon_terms(x)
    for t in range(3):
        assert _half_ulp_ok(y[t], y[t + 1])
    for k in range(300):
        assert sum(Fraction(float(v)) for v in x[:, k]) == sum(Fraction(float(v)) for v in y[:, k])
    # a canonical expansion is left as it is
    assert np.array_equal(I._canon_terms(y), y)


def test_rowcol_scaled_recipes():
    A, B = I.dd_rowcol_scaled(20, 30, 25, seed=9)
    A0, B0 = I.dd_random(20, 30, 10), I.dd_random(30, 25, 11)
    # each row of A (column of B) is one power of two times the unscaled matrix
    ra = np.log2(A[0] / A0[0])
    cb = np.log2(B[0] / B0[0])
    assert np.all(ra == ra[:, :1]) and np.all(cb == cb[:1, :])
    assert np.all(np.abs(ra) <= 16) and np.all(np.abs(cb) <= 16)
    assert np.array_equal(A[1], np.ldexp(A0[1], ra.astype(int))) and np.array_equal(B[1], np.ldexp(B0[1], cb.astype(int)))
    Q, R = I.qd_rowcol_scaled(8, 9, 7, seed=4)
    rq = np.log2(Q[0] / I.qd_random(8, 9, 5)[0])
    assert np.all(rq == rq[:, :1]) and np.all(np.abs(rq) <= 16)


def test_integer_matrices_are_exact_in_every_format():
    v = I.int_matrix(7, 5, 3, lo=-1000, hi=1000)
    assert v.min() >= -1000 and v.max() <= 1000
    assert np.array_equal(I.ints_to_dd(v)[0], v) and not I.ints_to_dd(v)[1].any()
    assert np.array_equal(I.ints_to_qd(v)[0], v) and not I.ints_to_qd(v)[1:].any()
    v[0, 0] = 0
    for w in (1, 2, 8):
        Y = I.ints_to_mp(v, w)
        for idx, x in enumerate(v.reshape(-1).tolist()):
            assert _mp_value(Y, w, idx) == x
        assert int(Y[1, 0, 0]) == 2                         # +0


def _isqrt_value(c, k, F=400):
    return Fraction(math.isqrt(c * k * k << (2 * F)), 1 << F)


@pytest.mark.parametrize("fmt,T", [("dd", 2), ("qd", 4)])
def test_paper_matrices_are_rounded_square_roots(fmt, T):
    # A = [sqrt(5)(i + j - 1)], B = [sqrt(3)(n - i)] (Section 4), as the greedy
    # T-term rounding: the remainder after T terms is below 2^-(53 T - 4) of
    # the value
    n = 9
    A, B = I.paper_matrices(n, fmt)
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            for X, c, k in ((A, 5, i + j - 1), (B, 3, n - i)):
                got = sum(Fraction(float(t)) for t in X[:, i - 1, j - 1])
                true = _isqrt_value(c, k)
                assert abs(got - true) <= (true + 1) * Fraction(1, 2 ** (53 * T - 4))
    # B's last row is zero (n - i = 0)
    assert not B[:, n - 1, :].any()


@pytest.mark.parametrize("w", [2, 8])
def test_paper_matrices_multi_limb(w):
    n = 6
    A, B = I.paper_matrices(n, "mp", w)
    p = 32 * w
    for idx in range(n * n):
        i, j = divmod(idx, n)
        a = _mp_value(A, w, idx)
        true = _isqrt_value(5, i + j + 1, F=2 * p)
        assert abs(a - true) <= true * Fraction(1, 2 ** p)   # RN to p bits: half an ulp
    assert all(int(v) == 2 for v in B[1, n - 1, :])           # sqrt(3)(n - n) = +0


def test_paper_closed_form():
    n = 7
    for i in range(1, n + 1):
        assert I.paper_closed_form(n, i) == sum((i + k - 1) * (n - k) for k in range(1, n + 1))


def test_batched_shapes_recipe():
    S = I.batched_shapes()
    assert len(S) == 512 and S == I.batched_shapes()
    dims = np.array([s[:3] for s in S])
    assert dims.min() >= 16 and dims.max() <= 1024
    # log-uniform: the median near sqrt(16 * 1024) = 128, a quarter below 45
    assert 90 < np.median(dims) < 180
    assert 0.15 < np.mean(dims < 45) < 0.35
    kinds = [s[3] for s in S]
    assert set(kinds) == {"dd", "qd", "mp256"} and min(kinds.count(k) for k in set(kinds)) > 130
