"""The high-part ("short") product rule of the GPU multi-limb multiply,
checked in exact integer arithmetic on the host.

For W >= 8 limbs the device sums only the limb products x_i y_j with
i + j >= W - 2.  The rule it relies on: the dropped products add less than
W units of limb W - 1, so when limb W - 1's bits below the kept mantissa M
lie more than W + 1 units from the half-ulp and from the next ulp, M and the
round-to-nearest-even increment taken from the partial sum are those of the
exact product; otherwise the device forms the full product.  This test
restates the rule with Python integers, asserts the error bound, and checks
every decided case against RNE of the exact product, on uniform mantissas
and on the structured ones (runs of zeros and ones, ties) that drive the
undecided branch.
"""

import numpy as np
import pytest

from paper_1710_01839_gb300 import inputs as I


def _mantissas(planes, w):
    limbs = planes[2:].reshape(w, -1).astype(object)
    return [sum(int(limbs[q, k]) << (32 * q) for q in range(w)) for k in range(limbs.shape[1])]


def _rne_exact(x, y, w):
    """(M, sh, carry) of RN_p(x y), p = 32 w, M before the carry is folded."""
    p = 32 * w
    t = x * y
    sh = 2 * p - t.bit_length()            # 0 or 1: t in [2^(2p-2), 2^(2p))
    drop = p - sh
    m, rest = t >> drop, t & ((1 << drop) - 1)
    half = 1 << (drop - 1)
    inc = rest > half or (rest == half and (m & 1))
    return m + int(inc), sh


def _short_rule(x, y, w):
    """The device's decision from the high part: (M + inc, sh) or None."""
    mask = (1 << 32) - 1
    part = 0
    for i in range(w):
        j0 = max(0, w - 2 - i)
        xi = (x >> (32 * i)) & mask
        part += (xi * (y >> (32 * j0))) << (32 * (i + j0))
    exact = x * y
    assert 0 <= exact - part < w * (1 << (32 * (w - 1)))    # the dropped products' bound
    sh = 0 if (part >> (64 * w - 1)) & 1 else 1
    ulp1 = 0x7FFFFFFF if sh else 0xFFFFFFFF
    half = 0x40000000 if sh else 0x80000000
    u = (part >> (32 * (w - 1))) & ulp1
    if u <= half - (w + 1) or (half < u <= ulp1 - w):
        m = part >> (32 * w - sh)
        return m + int(u > half), sh
    return None


@pytest.mark.parametrize("w", [4, 8, 16, 32, 64])
def test_short_product_rule_matches_exact_rounding(w):
    n = 600 if w <= 16 else 200
    decided = {"uniform": 0, "structured": 0}
    undecided = {"uniform": 0, "structured": 0}
    for kind, gen in (("uniform", I.mp_random), ("structured", I.mp_structured)):
        xs = _mantissas(gen(1, n, w, 9100 + w), w)
        ys = _mantissas(gen(1, n, w, 9200 + w), w)
        for x, y in zip(xs, ys):
            got = _short_rule(x, y, w)
            if got is None:
                undecided[kind] += 1
            else:
                decided[kind] += 1
                assert got == _rne_exact(x, y, w)
    # uniform mantissas are decided by the high part; the structured ones
    # reach both branches (at 32 and 64 limbs too rarely for this sample:
    # test_short_product_rule_ties covers them)
    assert undecided["uniform"] == 0
    assert decided["structured"] > 0
    if w <= 16:
        assert undecided["structured"] > 0


def test_short_product_rule_boundaries():
    # products placed just inside and just outside the decided windows
    w = 4
    p = 32 * w
    rng = np.random.default_rng(77)
    hits = 0
    for _ in range(3000):
        x = (1 << (p - 1)) | int(rng.integers(0, 1 << 62)) << 40 | int(rng.integers(0, 1 << 31))
        y = (1 << (p - 1)) | int(rng.integers(0, 1 << 62)) << 40 | int(rng.integers(0, 1 << 31))
        got = _short_rule(x, y, w)
        if got is not None:
            hits += 1
            assert got == _rne_exact(x, y, w)
    assert hits > 0


@pytest.mark.parametrize("w", [4, 8, 16, 32, 64])
def test_short_product_rule_ties(w):
    p = 32 * w
    # exact products (nothing below M) are decided, as rounding down
    for x, y in (((1 << (p - 1)), (1 << (p - 1))), ((1 << (p - 1)) + 1, 1 << (p - 1))):
        assert _short_rule(x, y, w) == _rne_exact(x, y, w)
    # an exact tie, (2^(p-1) + 1) 3 2^(p-2) = 3 2^(2p-3) + 2^(p-1) + 2^(p-2), is left open
    x, y = (1 << (p - 1)) + 1, 3 << (p - 2)
    assert _short_rule(x, y, w) is None
    # so are products one unit either side of the tie and just below the next ulp
    for x, y in (((1 << (p - 1)) + 3, 3 << (p - 2)), ((1 << p) - 1, (1 << p) - 1)):
        assert _short_rule(x, y, w) is None or _short_rule(x, y, w) == _rne_exact(x, y, w)
