"""The rules behind the DD / QD kernels' integer-pipe error terms, restated
with Python integers and checked against exact rational arithmetic.

TwoSum error (x with exponent field >= y's, s = RN(x + y), all normal,
e(x) - e(y) <= 54, s not below y's binade): x, y, s are integer multiples
of ulp(y) and |x + y - s| <= ulp(s)/2 < 2^55 ulp(y), so (x + y - s)/ulp(y)
equals the sum of the three scaled mantissas taken modulo 2^64.

TwoProd (a, b normal, exponent fields summing to 1129..3067, i.e. products
from 2^-917 up to below 2^1023): P = Ma Mb from four
32 x 32-bit products of the mantissas' 21- and 32-bit halves, shifted left
by 0 or 1 into [2^105, 2^106); p's mantissa is P / 2^53 rounded to nearest
even from the guard bit 52 and the sticky bits 0-51 (a carry to 2^53 goes
into the exponent field by packing (E - 1) 2^52 + q), and e = P - q 2^53 =
(P mod 2^53) - up 2^53, |e| <= 2^52 units.  The model below follows the
kernel's 32-bit words and funnel shifts step by step.

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


M32 = (1 << 32) - 1


def _funnel_l(lo, hi, n):
    return ((((hi << 32) | lo) << n) >> 32) & M32


def _funnel_r(lo, hi, n):
    return (((hi << 32) | lo) >> n) & M32


def exact_to_double(eu, ge):
    """The double eu 2^ge (|eu| <= 2^53, no rounding), None if subnormal."""
    if eu == 0:
        return 0.0
    m = abs(eu)
    lz = 64 - m.bit_length()
    F = 63 - lz + ge + 1023
    if F <= 0:
        return None
    mant = m << (lz - 11) if lz >= 11 else m >> (11 - lz)
    return from_bits(((1 << 63) if eu < 0 else 0) + ((F - 1) << 52) + mant)


def two_prod_int(a, b):
    """(p, e) as the kernel's integer-pipe TwoProd computes them, or None
    where it takes __dmul_rn and the FMA."""
    ba, bb = bits(a), bits(b)
    ah, al, bh, bl = ba >> 32, ba & M32, bb >> 32, bb & M32
    Ea, Eb = (ah >> 20) & 0x7FF, (bh >> 20) & 0x7FF
    if not (1 <= Ea <= 0x7FE and 1 <= Eb <= 0x7FE and 1129 <= Ea + Eb <= 3067):
        return None
    a1, b1 = (ah & 0xFFFFF) | 0x100000, (bh & 0xFFFFF) | 0x100000
    p00 = al * bl
    mid = al * b1 + a1 * bl
    assert mid < 1 << 54
    t = (p00 >> 32) + (mid & M32)
    u = a1 * b1 + (mid >> 32) + (t >> 32)
    w0, w1, w2, w3 = p00 & M32, t & M32, u & M32, u >> 32
    assert (w3 << 96 | w2 << 64 | w1 << 32 | w0) == ((ba & MM) | 1 << 52) * ((bb & MM) | 1 << 52)
    top = w3 >> 9
    sh = 1 - top
    w3, w2, w1, w0 = _funnel_l(w2, w3, sh), _funnel_l(w1, w2, sh), _funnel_l(w0, w1, sh), (w0 << sh) & M32
    qlo, qhi = _funnel_r(w1, w2, 21), _funnel_r(w2, w3, 21)
    up = (w1 >> 20) & (1 if ((w1 & 0xFFFFF) | w0) else qlo) & 1
    q = ((qhi << 32) | qlo) + up
    Ep = Ea + Eb - 1023 + top
    sgn = (ah ^ bh) & 0x80000000
    phi = sgn | ((((Ep - 1) << 20) + (q >> 32)) & M32)
    p = from_bits((phi << 32) | (q & M32))
    v = to_signed((((w1 & 0x1FFFFF) << 32) | w0) - (up << 53))
    assert abs(v) <= 1 << 52
    e = exact_to_double(-v if sgn else v, Ea + Eb - 2150 - sh)
    if e is None:
        return None
    return p, e


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


def _check_two_prod(a, b):
    r = two_prod_int(a, b)
    if r is None:
        return False
    p, e = r
    assert bits(p) == bits(a * b)                          # the IEEE product, bit for bit
    assert Fraction(a) * Fraction(b) == Fraction(p) + Fraction(e)
    return True


def test_two_prod_rule_is_the_exact_error():
    rng = np.random.default_rng(5)
    a_s, b_s = _doubles(rng, 5000, -500, 500), _doubles(rng, 5000, -500, 500)
    for a, b in zip(a_s, b_s):
        if not _check_two_prod(a, b):                  # outside [2^-917, 2^1022): FP64
            assert abs(a * b) < 2.0 ** -915
    # products near the range's edges (exponent fields summing to 1129..3067:
    # products from 2^-917, and below 2^1023)
    for a, b, want in ((2.0 ** -458, 2.0 ** -459, True), (2.0 ** -459, 2.0 ** -459, False),
                       (2.0 ** 511, 2.0 ** 510, True), (1.5 * 2.0 ** 511, 1.5 * 2.0 ** 510, True),
                       (1.99 * 2.0 ** 511, 1.99 * 2.0 ** 510, True), (2.0 ** 511, 2.0 ** 511, False)):
        assert _check_two_prod(a, b) == want
        assert 2.0 ** -917 <= abs(a * b) < 2.0 ** 1023 or not want
    # products that round up into the next binade, exact ones, and ties
    u = 2.0 ** -53
    for a, b in ((1 + 2 * u, 2 - 2 * u), (math.sqrt(2.0), math.sqrt(2.0)), (2 - 2 * u, 2 - 2 * u), (3.0, 0.5),
                 (1.0, 1.0), (-1.5, 1 + 4 * u)):
        assert _check_two_prod(a, b)
    for k in range(1, 200, 2):       # P < 2^105, P mod 2^52 = 2^51: ties, both parities of q
        assert _check_two_prod(1.5, 1 + k * 2 * u)
    for j in range(100):             # P >= 2^105, P mod 2^53 = 2^52
        assert _check_two_prod(1.75, ((5 << 50) + 4 + 8 * j) * 2.0 ** -52)
    carried = 0
    for _ in range(3000):
        x = int(rng.integers(1 << 52, 1 << 53))
        for top in (106, 105):
            y = ((1 << top) - 1) // x
            if (1 << 52) <= y < (1 << 53):
                a, b = x * 2.0 ** -52, y * 2.0 ** -52
                assert _check_two_prod(a, b)
                carried += a * b in (2.0, 4.0)
    assert carried > 100
    # zeros, subnormals, infinities, NaN and out-of-range products take FP64
    for a, b in ((0.0, 1.0), (2.0 ** -1074, 1.0), (math.inf, 1.0), (math.nan, 1.0), (2.0 ** -600, 2.0 ** -600),
                 (2.0 ** 600, 2.0 ** 600)):
        assert two_prod_int(a, b) is None


# ---------------------------------------------------------------- the Strassen passes' DD addition
#
# Every error term on the integer pipe (sum_err_int / two_sum_int /
# fast_two_sum_int / dd_add_int of the device header), with no FP64
# fallback: zeros are exact (y = +-0 gives r = y, s = +-0 with y != 0 gives
# +0, as y - (s - x) does), and the cases that need the FP64 formula set a
# flag instead (the passes then recompute the element with FP64 error terms).

def sum_err_total(x, y, s):
    """(r, rare) for x with exponent field >= y's, s = RN(x + y)."""
    bx, by, bs = bits(x), bits(y), bits(s)
    Ex, Ey, Es = (bx >> 52) & 0x7FF, (by >> 52) & 0x7FF, (bs >> 52) & 0x7FF
    if Ex == 0x7FF or Es == 0x7FF:
        return None, True
    if Ey == 0:
        return (y, False) if (by << 1) & M64 == 0 else (None, True)
    dxy = Ex - Ey
    if dxy > 54:
        return y, False
    if Es < Ey:
        return 0.0, False
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
        return 0.0, False
    r = assemble(ri, Ey)
    return (None, True) if r is None else (r, False)


def two_sum_int_model(a, b):
    x, y = _ordered(a, b)
    s = x + y
    e, rare = sum_err_total(x, y, s)
    return s, e, rare


def fast_two_sum_int_model(a, b):
    s = a + b
    Ea, Eb = (bits(a) >> 52) & 0x7FF, (bits(b) >> 52) & 0x7FF
    if Ea >= Eb:
        e, rare = sum_err_total(a, b, s)
        return s, e, rare
    return s, 0.0, Eb == 0x7FF or (bits(a) << 1) & M64 != 0


def dd_add_int_model(xh, xl, yh, yl, all_int=False):
    """dd_add_int: the first Fast2Sum by its FP64 formula, the other three
    error terms by the integer rule (all_int: all four, the form that ran
    6 FP64 operations per addition)."""
    sh, sl, r1 = two_sum_int_model(xh, yh)
    th, tl, r2 = two_sum_int_model(xl, yl)
    if r1 or r2:
        return None
    c = sl + th
    if all_int:
        vh, vl, r3 = fast_two_sum_int_model(sh, c)
        if r3:
            return None
    else:
        vh = sh + c
        vl = c - (vh - sh)
    w = tl + vl
    zh, zl, r4 = fast_two_sum_int_model(vh, w)
    return None if r4 else (zh, zl)


def dd_add_fp64(xh, xl, yh, yl):
    """The kernels' dd_add with FP64 error terms: TwoSum as Fast2Sum after
    ordering by exponent field, then the accurate double-word steps."""
    def two_sum(a, b):
        x, y = _ordered(a, b)
        s = x + y
        return s, y - (s - x)

    def fast_two_sum(a, b):
        s = a + b
        return s, b - (s - a)

    sh, sl = two_sum(xh, yh)
    th, tl = two_sum(xl, yl)
    vh, vl = fast_two_sum(sh, sl + th)
    return fast_two_sum(vh, tl + vl)


def _same(p, q):
    return all(bits(a) == bits(b) for a, b in zip(p, q))


@pytest.mark.parametrize("all_int", [False, True])
def test_dd_add_int_rule_on_dd_pairs(all_int):
    rng = np.random.default_rng(71)
    n = 4000
    hi = rng.uniform(-1, 1, (4, n)) * np.ldexp(1.0, rng.integers(-20, 21, (4, n)))
    lo = np.ldexp(hi, -53) * rng.uniform(-1, 1, (4, n))
    for i in range(n):
        xh, yh = float(hi[0, i]), float(hi[1, i])
        xl, yl = float(lo[0, i]), float(lo[1, i])
        for sgn in (1.0, -1.0):
            z = dd_add_int_model(xh, xl, sgn * yh, sgn * yl, all_int)
            assert z is not None                    # none of these is rare
            assert _same(z, dd_add_fp64(xh, xl, sgn * yh, sgn * yl))


@pytest.mark.parametrize("all_int", [False, True])
def test_dd_add_int_rule_on_cancellations(all_int):
    rng = np.random.default_rng(72)
    flagged = 0
    for k in range(-3, 4):
        for _ in range(400):
            xh = float(rng.uniform(-1, 1)) * 2.0 ** int(rng.integers(-30, 30))
            xl = math.ldexp(xh, -53) * float(rng.uniform(-1, 1))
            yh = -(xh + k * math.ulp(xh))
            yl = -xl * float(rng.uniform(0.25, 4)) * float(rng.choice([-1, 1]))
            z = dd_add_int_model(xh, xl, yh, yl, all_int)
            if z is None:
                flagged += 1
                continue
            assert _same(z, dd_add_fp64(xh, xl, yh, yl))
            # the exact sum's error: the accurate addition's bound 3u^2 |x + y|
            exact = Fraction(xh) + Fraction(xl) + Fraction(yh) + Fraction(yl)
            assert abs(Fraction(z[0]) + Fraction(z[1]) - exact) <= 3 * Fraction(2) ** -106 * abs(exact)
    assert flagged < (7 * 400 if all_int else 70)     # the kept form seldom flags a cancellation


@pytest.mark.parametrize("all_int", [False, True])
def test_dd_add_int_rule_special_values(all_int):
    u = 2.0 ** -53
    vals = [0.0, -0.0, 1.0, -1.0, 1 + 2 * u, u, 2.0 ** -1074, 2.0 ** -1022, 1.7976931348623157e308, math.inf,
            -math.inf, math.nan, 2.0 ** -1000, 3.0]
    unflagged = 0
    for xh in vals:
        for xl in vals:
            for yh in vals:
                for yl in vals:
                    z = dd_add_int_model(xh, xl, yh, yl, all_int)
                    if not all(math.isfinite(v) for v in (xh, xl, yh, yl)):
                        assert z is None            # every infinity and NaN is flagged
                    if z is None:
                        continue
                    unflagged += 1
                    assert _same(z, dd_add_fp64(xh, xl, yh, yl))
    assert unflagged > 5000
