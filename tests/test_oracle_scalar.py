"""Pins of the oracle's scalar arithmetic against exact rational arithmetic
and mpmath (no GPU).

* TwoSum / Fast2Sum / TwoProd: s + e == a + b (a * b) exactly, s = RN(a + b).
* DD add / multiply: relative error within the published double-word bounds
  (3u^2 and 5u^2), result non-overlapping.
* QD add / multiply: bit-identical to the exact result rounded greedily to
  four doubles (computed with Fractions).
* Multi-limb add / multiply: bit-identical to mpmath's correctly rounded
  mpf_add / mpf_mul (round-nearest-even) and to a Fraction-based RNE; ties,
  carry-out and cancellation constructed explicitly.
"""

import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact import (F, U, greedy, mp_from_mpmath, mp_round_fraction, mp_words, mp_words_to_fraction,
                   non_overlapping, ulp, value)


def _rand_doubles(rng, n, emin=-60, emax=60):
    m = rng.uniform(0.5, 1.0, size=n) * rng.choice([-1.0, 1.0], size=n)
    e = rng.integers(emin, emax, size=n)
    return np.ldexp(m, e)


EDGE_PAIRS = [
    (1.0, -1.0), (1.0, 2.0**-60), (2.0**53, 1.0), (2.0**53, -1.0), (0.0, 3.5), (-0.0, 0.0),
    (1.0 + 2.0**-52, -1.0), (3.0, 2.0**-53 * 3), (1e300, -1e300 * (1 - 2.0**-52)), (0.1, 0.2),
]


# ------------------------------------------------------------------ EFTs

def test_two_sum_exact():
    rng = np.random.default_rng(1)
    a = _rand_doubles(rng, 4000)
    b = _rand_doubles(rng, 4000)
    pairs = list(zip(a.tolist(), b.tolist())) + EDGE_PAIRS
    for x, y in pairs:
        s, e = oracle.two_sum(x, y)
        assert s == float(F(x) + F(y))
        assert F(s) + F(e) == F(x) + F(y)


def test_fast_two_sum_exact_when_ordered():
    rng = np.random.default_rng(2)
    a = _rand_doubles(rng, 4000)
    b = _rand_doubles(rng, 4000)
    for x, y in list(zip(a.tolist(), b.tolist())) + EDGE_PAIRS:
        if abs(x) < abs(y):
            x, y = y, x
        s, e = oracle.fast_two_sum(x, y)
        assert F(s) + F(e) == F(x) + F(y)


def test_two_prod_exact():
    rng = np.random.default_rng(3)
    a = _rand_doubles(rng, 4000)
    b = _rand_doubles(rng, 4000)
    for x, y in list(zip(a.tolist(), b.tolist())) + EDGE_PAIRS[:8]:
        p, e = oracle.two_prod(x, y)
        assert p == float(F(x) * F(y))
        assert F(p) + F(e) == F(x) * F(y)


def _scaled(x: float) -> int:
    """x * 2^1074 as an exact integer (every finite double is a multiple of
    2^-1074)."""
    num, den = x.as_integer_ratio()
    return num << (1075 - den.bit_length())


@pytest.mark.slow
@pytest.mark.parametrize("op", ["two_sum", "fast_two_sum", "two_prod"])
def test_error_free_transformations_on_a_million_pairs(op):
    # exact integer arithmetic at the scale 2^1074: s + e == a + b (a * b),
    # s (p) the IEEE round-to-nearest sum (product) that numpy computes
    rng = np.random.default_rng({"two_sum": 11, "fast_two_sum": 12, "two_prod": 13}[op])
    n = 1_000_000
    a = _rand_doubles(rng, n, -60, 60)
    b = _rand_doubles(rng, n, -60, 60)
    if op == "fast_two_sum":
        swap = np.abs(a) < np.abs(b)
        a, b = np.where(swap, b, a), np.where(swap, a, b)
    f = getattr(oracle, op)
    ref = a * b if op == "two_prod" else a + b
    for x, y, r in zip(a.tolist(), b.tolist(), ref.tolist()):
        s, e = f(x, y)
        assert s == r
        if op == "two_prod":
            assert _scaled(x) * _scaled(y) == (_scaled(s) + _scaled(e)) << 1074
        else:
            assert _scaled(x) + _scaled(y) == _scaled(s) + _scaled(e)


# ------------------------------------------------------------------ DD

def _rand_dd(rng, n, emin=-30, emax=30):
    # lo = U(-1/2, 1/2) ulp(hi) 2^-j: numpy's uniform doubles sit on a fixed
    # 2^-53 grid, so without the random shift j every sum of two lo parts
    # would be exact and a dropped rounding-error term would go unseen
    out = []
    for _ in range(n):
        hi = float(_rand_doubles(rng, 1, emin, emax)[0])
        lo = float(rng.uniform(-0.5, 0.5)) * float(ulp(hi)) * 2.0 ** -int(rng.integers(0, 12))
        out.append((hi, lo))
    return out


def test_dd_add_error_bound_and_normalised():
    rng = np.random.default_rng(4)
    xs = _rand_dd(rng, 3000)
    ys = _rand_dd(rng, 3000)
    # cancellation-heavy pairs: y close to -x, the low parts at other exponents
    # (their sum is then rarely a double, and the result is that sum as a DD)
    for i in range(500):
        hi, lo = xs[i]
        ys[i] = (-hi, float(rng.uniform(-0.5, 0.5)) * float(ulp(hi)) * 2.0 ** -int(rng.integers(1, 12)))
    worst = Fraction(0)
    for x, y in zip(xs, ys):
        z = oracle.dd_add(x, y)
        ex = value(x) + value(y)
        assert non_overlapping(z.tolist())
        if ex == 0:
            assert value(z) == 0
            continue
        rel = abs(value(z) - ex) / abs(ex)
        worst = max(worst, rel)
    assert worst <= 3 * U * U * (1 + 8 * U), float(worst / (U * U))


def test_dd_mul_error_bound_and_normalised():
    rng = np.random.default_rng(5)
    xs = _rand_dd(rng, 3000)
    ys = _rand_dd(rng, 3000)
    worst = Fraction(0)
    for x, y in zip(xs, ys):
        z = oracle.dd_mul(x, y)
        ex = value(x) * value(y)
        assert non_overlapping(z.tolist())
        rel = abs(value(z) - ex) / abs(ex)
        worst = max(worst, rel)
    assert worst <= 5 * U * U, float(worst / (U * U))
    # a dropped xl*yl or cross term would show up far above u^2 on these
    assert worst > 0


# ------------------------------------------------------------------ QD

def _rand_qd(rng, n):
    out = []
    for _ in range(n):
        x0 = float(_rand_doubles(rng, 1, -20, 20)[0])
        t = [x0]
        for _ in range(3):
            t.append(float(rng.uniform(-0.5, 0.5)) * float(ulp(t[-1])) if t[-1] != 0 else 0.0)
        out.append(greedy(value(t), 4))
    return out


def test_qd_add_is_exact_rounded():
    rng = np.random.default_rng(6)
    xs = _rand_qd(rng, 600)
    ys = _rand_qd(rng, 600)
    for i in range(100):
        ys[i] = [-v for v in xs[i]]             # total cancellation
    for i in range(100, 200):
        ys[i] = [-xs[i][0], xs[i][1], 0.0, 0.0]  # partial cancellation
    for x, y in zip(xs, ys):
        z = oracle.qd_add(x, y)
        assert z.tolist() == greedy(value(x) + value(y), 4)


def test_qd_mul_is_exact_rounded_and_bounded():
    rng = np.random.default_rng(7)
    xs = _rand_qd(rng, 600)
    ys = _rand_qd(rng, 600)
    for x, y in zip(xs, ys):
        z = oracle.qd_mul(x, y)
        ex = value(x) * value(y)
        assert z.tolist() == greedy(ex, 4)
        assert abs(value(z) - ex) <= abs(ex) * 2 * U**4


def test_round_terms_matches_greedy():
    rng = np.random.default_rng(8)
    for _ in range(300):
        v = _rand_doubles(rng, 12, -150, 150)
        for T in (1, 2, 4):
            assert oracle.round_terms(v, T).tolist() == greedy(sum(F(x) for x in v), T)


# ------------------------------------------------------------------ multi-limb

def _rand_mp(rng, w, emin=-64, emax=64):
    p = 32 * w
    M = (1 << (p - 1)) | rng.getrandbits(p - 1)
    return rng.randint(emin, emax), rng.randint(0, 1), M


def _to_mpf(e, s, M, w):
    from mpmath.libmp import from_man_exp
    return from_man_exp(-M if s else M, e - 32 * w)


def _check_against_refs(w, x, y, op):
    from mpmath.libmp import mpf_add, mpf_mul
    p = 32 * w
    xw, yw = mp_words(*x, w), mp_words(*y, w)
    if op == "mul":
        got = oracle.mp_mul(w, xw, yw)
        ex = mp_words_to_fraction(xw, w) * mp_words_to_fraction(yw, w)
        ref = mpf_mul(_to_mpf(*x, w), _to_mpf(*y, w), p, "n")
    else:
        got = oracle.mp_add(w, xw, yw)
        ex = mp_words_to_fraction(xw, w) + mp_words_to_fraction(yw, w)
        ref = mpf_add(_to_mpf(*x, w), _to_mpf(*y, w), p, "n")
    want = mp_round_fraction(ex, w)
    assert mp_from_mpmath(ref, w) == want
    assert got.tolist() == mp_words(*want, w).tolist(), (x, y, op)


@pytest.mark.parametrize("w", [1, 2, 4, 8, 32, 64])
def test_mp_random_vs_mpmath(w):
    pytest.importorskip("mpmath")
    rng = random.Random(100 + w)
    n = 400 if w <= 8 else 120 if w <= 32 else 60
    for _ in range(n):
        x, y = _rand_mp(rng, w), _rand_mp(rng, w)
        _check_against_refs(w, x, y, "mul")
        _check_against_refs(w, x, y, "add")
        # close exponents force deep cancellation / alignment paths
        y2 = (x[0] + rng.randint(-2, 2), 1 - x[1], y[2])
        _check_against_refs(w, x, y2, "add")


@pytest.mark.slow
@pytest.mark.parametrize("w,n", [(1, 100_000), (2, 100_000), (4, 100_000), (8, 100_000)])
def test_mp_many_random_pairs_vs_mpmath(w, n):
    # mpmath's correctly rounded mpf_mul / mpf_add alone (the Fraction
    # reference is left to the smaller test above), on n random pairs per
    # width, with exponents close enough for every alignment and
    # cancellation depth
    pytest.importorskip("mpmath")
    from mpmath.libmp import mpf_add, mpf_mul
    p = 32 * w
    rng = random.Random(7000 + w)
    for _ in range(n):
        x = _rand_mp(rng, w, -4, 4)
        y = (rng.randint(x[0] - p - 3, x[0] + 2), rng.randint(0, 1), (1 << (p - 1)) | rng.getrandbits(p - 1))
        xw, yw = mp_words(*x, w), mp_words(*y, w)
        fx, fy = _to_mpf(*x, w), _to_mpf(*y, w)
        assert oracle.mp_mul(w, xw, yw).tolist() == mp_words(*mp_from_mpmath(mpf_mul(fx, fy, p, "n"), w), w).tolist()
        assert oracle.mp_add(w, xw, yw).tolist() == mp_words(*mp_from_mpmath(mpf_add(fx, fy, p, "n"), w), w).tolist()


@pytest.mark.parametrize("w", [1, 4, 64])
def test_mp_constructed_ties_and_carries(w):
    pytest.importorskip("mpmath")
    p = 32 * w
    half = 1 << (p - 1)
    cases = []
    # add: x + half an ulp of x, x with odd and even mantissa -> ties both ways
    for M in (half + 1, half + 2, (1 << p) - 1, half):
        cases.append(((10, 0, M), (10 - p, 0, half), "add"))        # y = 2^(10-p-1) = ulp/2
        cases.append(((10, 0, M), (10 - p, 1, half), "add"))
    # carry-out to 2^p
    cases.append((((7, 0, (1 << p) - 1)), (7 - p, 0, half + 1), "add"))
    # exact cancellation, and x - tiny at a power of two
    cases.append(((3, 0, half + 5), (3, 1, half + 5), "add"))
    cases.append(((3, 0, half), (3 - p - 1, 1, half + 3), "add"))
    cases.append(((3, 0, half), (3 - p - 5, 1, half + 3), "add"))
    cases.append(((3, 0, half), (3 - 2 * p, 1, half), "add"))
    # multiply ties: M_x = 3*2^(p-2), M_y = 2^(p-1)+1 gives a round bit of 1 and no sticky
    cases.append(((1, 0, 3 << (p - 2)), (1, 0, half + 1), "mul"))
    cases.append(((1, 1, 3 << (p - 2)), (1, 0, half + 3), "mul"))
    cases.append(((1, 0, (1 << p) - 1), (1, 0, (1 << p) - 1), "mul"))
    for x, y, op in cases:
        _check_against_refs(w, x, y, op)


def test_mp_zero_rules():
    w = 2
    z = mp_words(0, 0, 0, w)
    nz = mp_words(0, 1, 0, w)
    x = mp_words(5, 1, (1 << 63) | 12345, w)
    assert oracle.mp_add(w, z, x).tolist() == x.tolist()
    assert oracle.mp_add(w, x, z).tolist() == x.tolist()
    assert oracle.mp_add(w, z, nz).tolist() == z.tolist()             # +0 + -0 = +0
    assert oracle.mp_add(w, nz, nz).tolist() == nz.tolist()           # -0 + -0 = -0
    assert oracle.mp_mul(w, x, z).tolist() == nz.tolist()             # (-x) * (+0) = -0
    negx = x.copy()
    negx[1] ^= 1
    assert oracle.mp_add(w, x, negx).tolist() == z.tolist()           # x + (-x) = +0
