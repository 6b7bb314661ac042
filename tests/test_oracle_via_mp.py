"""Pins of the oracle's conversions between DD / QD expansions and p-bit
multi-limb numbers (the DD / QD GEMM computed in multi-limb arithmetic),
against exact rational arithmetic written out here with Python integers:

  to p bits:   c = +0, c = RN_p(c + x_t) for t = 0..T-1;
  from p bits: x_t = RN_53(r), r = r - x_t (Python's float(Fraction) is the
               correctly rounded, ties-to-even double).
"""

from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1710_01839_gb300 import inputs as I


def rn_p(x: Fraction, p: int) -> Fraction:
    """x rounded to p significant bits, ties to even."""
    if x == 0:
        return Fraction(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    # a in [2^e, 2^(e+1)); scale so that p bits sit above the point
    scaled = a / Fraction(2) ** (e - p + 1)
    q, r = divmod(scaled.numerator, scaled.denominator)
    twice = 2 * r
    if twice > scaled.denominator or (twice == scaled.denominator and q % 2 == 1):
        q += 1
    return s * Fraction(q) * Fraction(2) ** (e - p + 1)


def mp_value(Y, w, idx):
    """Decode element idx of multi-limb planes to a Fraction."""
    e = int(Y[0].reshape(-1).view(np.int32)[idx])
    f = int(Y[1].reshape(-1)[idx])
    if f & 2:
        return Fraction(0), f & 1
    M = 0
    for q in range(w):
        M |= int(Y[2 + q].reshape(-1)[idx]) << (32 * q)
    assert M >> (32 * w - 1) == 1, "not normalised"
    v = Fraction(M) * Fraction(2) ** (e - 32 * w)
    return (-v if f & 1 else v), f & 1


def _check_to_mp(X, bits):
    T = X.shape[0]
    w = bits // 32
    Y = oracle.terms_to_mp(X, bits)
    for idx in range(X.shape[1] * X.shape[2]):
        c = Fraction(0)
        for t in range(T):
            c = rn_p(c + Fraction(float(X[t].reshape(-1)[idx])), bits)
        got, _ = mp_value(Y, w, idx)
        assert got == c, (idx, got, c)
    return Y


def _check_from_mp(Y, bits, T):
    w = bits // 32
    X = oracle.mp_to_terms(Y, bits, T)
    for idx in range(Y.shape[1] * Y.shape[2]):
        r, _ = mp_value(Y, w, idx)
        for t in range(T):
            x = float(r)
            assert X[t].reshape(-1)[idx] == x or (x == 0 and X[t].reshape(-1)[idx] == 0), (idx, t)
            r -= Fraction(x)
    return X


@pytest.mark.parametrize("bits", [64, 128, 256])
def test_dd_to_mp_is_rn_of_the_exact_sum(bits):
    X = I.dd_random(6, 7, 31 + bits, exp_spread=20)
    # lo pushed far below hi, so that hi + lo needs more than p bits
    X[1, :3] *= 2.0 ** -90
    _check_to_mp(X, bits)


@pytest.mark.parametrize("bits", [256, 512])
def test_qd_to_mp_is_sequential_rn(bits):
    X = I.qd_random(5, 6, 41 + bits, exp_spread=20)
    X[3, :2] *= 2.0 ** -200
    _check_to_mp(X, bits)


def test_to_mp_ties_and_zeros():
    bits = 64
    # 1 + 2^-64 is a tie at 64 bits (M = 2^63 even: stays 1); 1 + 3 2^-64 rounds
    # up; 1 - 2^-53 + 2^-65 is a tie that goes to the even neighbour 1 - 2^-53
    X = np.array([[[1.0, 1.0, 1.0 - 2.0 ** -53, -0.0, 0.0, 2.0 ** -1074]],
                  [[2.0 ** -64, 3 * 2.0 ** -64, 2.0 ** -65, -0.0, -0.0, 0.0]]])
    Y = _check_to_mp(X, bits)
    assert mp_value(Y, 2, 0)[0] == 1 and mp_value(Y, 2, 1)[0] == 1 + Fraction(2, 2 ** 63)
    assert mp_value(Y, 2, 2)[0] == 1 - Fraction(1, 2 ** 53)
    # zeros: the sum starts at +0 and +0 + -0 = +0 (the multi-limb add), so
    # all-zero expansions give +0
    assert int(Y[1, 0, 3]) == 2 and int(Y[1, 0, 4]) == 2


@pytest.mark.parametrize("bits,T", [(64, 2), (128, 2), (256, 4), (512, 4)])
def test_from_mp_is_the_greedy_expansion(bits, T):
    w = bits // 32
    Y = I.mp_random(5, 7, w, 77 + bits, emin=-300, emax=300)
    Y[2:, 0, 0] = 0
    Y[2 + w - 1, 0, 0] = 0x80000000         # a power of two
    Y[2:2 + w - 1, 0, 1] = 0xFFFFFFFF       # a run of ones below the top limb
    # halfway patterns for the first double: the bit below its 53 (index
    # p - 54) set and the bits under it clear in the top 64, then the lowest
    # bit of limb 0 set (above halfway: rounds up), clear (a tie: to even), and
    # an odd last bit with a clear tail (a tie: up to even)
    p = 32 * w
    for col, bit_list in ((2, [p - 1, p - 54, 0]), (3, [p - 1, p - 54]), (4, [p - 1, p - 53, p - 54])):
        M = sum(1 << b for b in bit_list)
        for q in range(w):
            Y[2 + q, 0, col] = (M >> (32 * q)) & 0xFFFFFFFF
        Y[1, 0, col] &= 1
    _check_from_mp(Y, bits, T)


def test_roundtrip_of_canonical_expansions():
    A = I.dd_random(8, 9, 5, exp_spread=20)
    assert np.array_equal(oracle.mp_to_terms(oracle.terms_to_mp(A, 128), 128, 2), A)
    Q = I.qd_random(8, 9, 6, exp_spread=20)
    assert np.array_equal(oracle.mp_to_terms(oracle.terms_to_mp(Q, 256), 256, 4), Q)


@pytest.mark.parametrize("algo,depth", [("simple", 0), ("block", 0), ("strassen", 2)])
def test_dd_gemm_via_mp_meets_a_128_bit_bound(algo, depth):
    # C within 2^-105 |C| (the final DD rounding) + (2 l + 4) 2^-128 |A||B|
    # of the exact product: two orders of magnitude inside the DD bound
    m, l, n = 12, 17, 10
    A = I.dd_random(m, l, 900, exp_spread=20)
    B = I.dd_random(l, n, 901, exp_spread=20)
    C = oracle.gemm_via_mp(A, B, 128, algo=algo, n_min=16, depth=depth)
    ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    err, absab = oracle.exact_check(A, B, C, ii.ravel(), jj.ravel())
    cabs = np.abs(C[0]).ravel()
    assert np.all(err <= 2.0 ** -105 * cabs + (2 * l + 4) * 2.0 ** -128 * absab)
    assert np.all(err <= 4 * l * 2.0 ** -104 * absab / 64)


def test_qd_gemm_via_mp_meets_a_256_bit_bound():
    m, l, n = 9, 11, 8
    A = I.qd_random(m, l, 910, exp_spread=20)
    B = I.qd_random(l, n, 911, exp_spread=20)
    C = oracle.gemm_via_mp(A, B, 256, algo="block", n_min=16)
    ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    err, absab = oracle.exact_check(A, B, C, ii.ravel(), jj.ravel())
    cabs = np.abs(C[0]).ravel()
    assert np.all(err <= 2.0 ** -210 * cabs + (2 * l + 4) * 2.0 ** -256 * absab)
