"""The rules behind the DD / QD kernels' integer-pipe error terms, restated
with Python integers and checked against exact rational arithmetic.

TwoSum error (x with exponent field >= y's, s = RN(x + y), all normal,
e(x) - e(y) <= 54, s not below y's binade): x, y, s are integer multiples
of ulp(y) and |x + y - s| <= ulp(s)/2 < 2^55 ulp(y), so (x + y - s)/ulp(y)
equals the sum of the three scaled mantissas taken modulo 2^64.

Product error (a, b, p = RN(a b) normal): the mantissa product Ma Mb and p's
mantissa scaled to the same unit (Mp 2^k, k = 52 or 53) differ by at most
2^52 units, so their difference is the low 64 bits of Ma Mb minus Mp 2^k
modulo 2^64.

Each function returns None where the kernels take the FP64 formula instead.
"""

import math
import struct
from fractions import Fraction

import numpy as np
import pytest

M64 = (1 << 64) - 1
MM = (1 << 52) - 1


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def from_bits(b):
    return struct.unpack("<d", struct.pack("<Q", b & M64))[0]


def to_signed(u):
    u &= M64
    return u - (1 << 64) if u >> 63 else u


def assemble(v, unit_field):
    """The double v * 2^(unit_field - 1075) for a nonzero integer |v| <= 2^55,
    or None when it would be subnormal; exact (v has <= 53 significant bits)."""
    m = abs(v)
    lz = 64 - m.bit_length()
    F = unit_field + 11 - lz
    if F <= 0:
        return None
    mant = m << (lz - 11) if lz >= 11 else m >> (11 - lz)
    assert (m >> (11 - lz)) << (11 - lz) == m if lz < 11 else True   # exact
    return from_bits(((1 << 63) if v < 0 else 0) | (F << 52) | (mant & MM))


def two_sum_err_int(x, y, s):
    bx, by, bs = bits(x), bits(y), bits(s)
    Ex, Ey, Es = (bx >> 52) & 0x7FF, (by >> 52) & 0x7FF, (bs >> 52) & 0x7FF
    if Ey == 0 or Ex == 0x7FF or Es == 0 or Es == 0x7FF:
        return None
    dxy = Ex - Ey
    if dxy > 54:
        return y
    if Es < Ey:
        return 0.0
    X = (((bx & MM) | (1 << 52)) << dxy) & M64
    Y = (by & MM) | (1 << 52)
    S = (((bs & MM) | (1 << 52)) << (Es - Ey)) & M64
    if bx >> 63:
        X = -X
    if by >> 63:
        Y = -Y
    if bs >> 63:
        S = -S
    ri = to_signed(X + Y - S)
    if ri == 0:
        return 0.0
    return assemble(ri, Ey)


def two_prod_err_int(a, b, p):
    ba, bb, bp = bits(a), bits(b), bits(p)
    Ea, Eb, Ep = (ba >> 52) & 0x7FF, (bb >> 52) & 0x7FF, (bp >> 52) & 0x7FF
    if 0 in (Ea, Eb, Ep) or 0x7FF in (Ea, Eb, Ep):
        return None
    Ma, Mb, Mp = (ba & MM) | (1 << 52), (bb & MM) | (1 << 52), (bp & MM) | (1 << 52)
    k = Ep - Ea - Eb + 1075
    assert k in (52, 53)
    eu = to_signed(Ma * Mb - (Mp << k))
    assert abs(eu) <= 1 << 52
    if eu == 0:
        return 0.0
    m = abs(eu)
    lz = 64 - m.bit_length()
    F = Ea + Eb - 1064 - lz
    if F <= 0:
        return None
    sgn = ((ba ^ bb) >> 63) ^ (1 if eu < 0 else 0)
    return from_bits((sgn << 63) | (F << 52) | ((m << (lz - 11)) & MM))


def _ordered(a, b):
    ea, eb = (bits(a) >> 52) & 0x7FF, (bits(b) >> 52) & 0x7FF
    return (b, a) if eb > ea else (a, b)


def _doubles(rng, n, emin=-1000, emax=1000):
    m = rng.uniform(1, 2, n) * rng.choice([-1.0, 1.0], n)
    return [float(v) for v in np.ldexp(m, rng.integers(emin, emax, n))]


@pytest.mark.parametrize("spread", [0, 2, 30, 53, 54, 55, 56, 200])
def test_two_sum_rule_is_the_exact_error(spread):
    rng = np.random.default_rng(spread)
    xs = _doubles(rng, 3000)
    used = 0
    for x0 in xs:
        y0 = x0 * float(rng.uniform(0.5, 2)) * 2.0 ** -int(rng.integers(0, spread + 1)) * float(rng.choice([-1, 1]))
        x, y = _ordered(x0, y0)
        s = x + y
        r = two_sum_err_int(x, y, s)
        if r is None:
            continue
        used += 1
        assert Fraction(x) + Fraction(y) == Fraction(s) + Fraction(r)
        assert bits(r) == bits(y - (s - x))        # bit for bit the FP64 formula (incl. +0)
    assert used > 2500


def test_two_sum_rule_edge_cases():
    u = 2.0 ** -53
    vals = [1.0, -1.0, 1 + 2 * u, 1 - u, 2.0, 3.0, 0.5, 2.0 ** -1022, 2.0 ** 1023, 1.5 * 2.0 ** -1000,
            2.0 ** -52, 2.0 ** -53, 2.0 ** -54, 2.0 ** -55, 3 * 2.0 ** -55, 0.0, -0.0, 2.0 ** -1074, math.inf]
    vals += [-v for v in vals]
    routed = 0
    for a in vals:
        for b in vals:
            x, y = _ordered(a, b)
            s = x + y
            r = two_sum_err_int(x, y, s)
            if r is None:
                routed += 1
                continue
            assert Fraction(x) + Fraction(y) == Fraction(s) + Fraction(r)
            assert bits(r) == bits(y - (s - x))
    assert routed > 0      # zeros, subnormals and infinities take the FP64 formula


def test_two_prod_rule_is_the_exact_error():
    rng = np.random.default_rng(5)
    a_s, b_s = _doubles(rng, 5000, -500, 500), _doubles(rng, 5000, -500, 500)
    for a, b in zip(a_s, b_s):
        p = a * b
        e = two_prod_err_int(a, b, p)
        if e is None:                              # e below the normal range: the FMA
            assert abs(p) < 2.0 ** -960
            continue
        assert Fraction(a) * Fraction(b) == Fraction(p) + Fraction(e)
    # products that round up into the next binade (k = 53) and exact ones
    u = 2.0 ** -53
    for a, b in ((1 + 2 * u, 2 - 2 * u), (math.sqrt(2.0), math.sqrt(2.0)), (2 - 2 * u, 2 - 2 * u), (3.0, 0.5),
                 (1.0, 1.0), (-1.5, 1 + 4 * u)):
        p = a * b
        e = two_prod_err_int(a, b, p)
        assert Fraction(a) * Fraction(b) == Fraction(p) + Fraction(e)
    # underflowing or overflowing products are routed to the FMA
    assert two_prod_err_int(2.0 ** -600, 2.0 ** -600, 2.0 ** -600 * 2.0 ** -600) is None
    assert two_prod_err_int(2.0 ** 600, 2.0 ** 600, math.inf) is None
