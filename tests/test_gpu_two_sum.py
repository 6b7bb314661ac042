"""The DD / QD kernels' TwoSum computes its error term on the integer pipe;
it must equal the FP64 formula y - (s - x) bit for bit for every pair of
doubles (mpgemm_selftest_two_sum runs both on the device).  Pairs: random
doubles over the whole exponent range, and crafted ones (equal exponents,
cancellation, powers of two, exponent gaps around 54, zeros of both signs,
subnormals, infinities, NaN, overflow), plus the accumulator / product
pairs of a DD multiply-accumulate.  The DD MAC's TwoProd (product and
error, both on the integer pipe; mpgemm_selftest_two_prod) must give the
host's IEEE product (numpy's float64 multiply) and the device FMA's error
bit for bit on the same kinds of pairs, plus products that round up into
the next binade, ties and products at the edges of the normal range."""

import numpy as np
import pytest

from gpu_util import dev

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")


def _run(a, b):
    import ctypes
    import torch
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = torch.empty(3 * len(a), dtype=torch.float64, device="cuda")
    ad, bd = dev(a), dev(b)
    rc = mpg.lib().mpgemm_selftest_two_sum(len(a), ctypes.c_void_p(ad.data_ptr()), ctypes.c_void_p(bd.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 0
    o = out.cpu().numpy().reshape(3, -1)
    return o[0], o[1], o[2]


def _bits(x):
    return np.ascontiguousarray(x).view(np.uint64)


def test_random_pairs_over_the_exponent_range():
    rng = np.random.default_rng(2024)
    n = 1 << 20
    bits = rng.integers(0, 2**63, size=(2, n), dtype=np.uint64) | (rng.integers(0, 2, size=(2, n), dtype=np.uint64) << np.uint64(63))
    a, b = bits[0].view(np.float64), bits[1].view(np.float64)
    s, e_int, e_fp = _run(a, b)
    assert np.array_equal(_bits(e_int), _bits(e_fp))


@pytest.mark.parametrize("spread", [0, 3, 20, 52, 53, 54, 55, 56, 60, 120])
def test_random_pairs_with_close_exponents(spread):
    # exponent gaps up to `spread`, both signs: rounding, cancellation, the
    # e(x) - e(y) > 54 shortcut and its boundary
    rng = np.random.default_rng(100 + spread)
    n = 1 << 18
    a = rng.uniform(1, 2, n) * np.ldexp(1.0, rng.integers(-900, 900, n))
    a *= rng.choice([-1.0, 1.0], n)
    b = rng.uniform(1, 2, n) * np.ldexp(a, -rng.integers(0, spread + 1, n)) * rng.choice([-1.0, 1.0], n)
    s, e_int, e_fp = _run(np.concatenate([a, b]), np.concatenate([b, a]))
    assert np.array_equal(_bits(e_int), _bits(e_fp))


def test_crafted_pairs():
    tiny = np.ldexp(1.0, -1074)
    big = np.finfo(np.float64).max
    u = 2.0 ** -53
    vals = [0.0, -0.0, 1.0, -1.0, 1.0 + 2 * u, 1.0 - u, 2.0, 3.0, 0.5, tiny, -tiny, 2 * tiny, np.ldexp(1.0, -1022),
            np.ldexp(1.0, -1022) * (1 - 2 * u), big, -big, np.inf, -np.inf, np.nan, np.ldexp(1.0, 1023),
            1.0 + u, np.ldexp(1.0, -52), np.ldexp(1.0, -53), np.ldexp(1.0, -54), np.ldexp(1.0, -55),
            np.ldexp(1.0, -56), np.ldexp(3.0, -55), np.ldexp(1.0, -1000), np.ldexp(1.0, 1000), 1e-300, 1e300]
    vals = np.array(vals + [-v for v in vals])
    a, b = np.meshgrid(vals, vals, indexing="ij")
    s, e_int, e_fp = _run(a.ravel(), b.ravel())
    assert np.array_equal(_bits(e_int), _bits(e_fp))


def test_multiply_accumulate_pairs():
    # (accumulator, product) pairs of DD GEMMs on the benchmark's inputs
    from paper_1710_01839_gb300 import inputs as I
    A = I.dd_random(64, 256, 5, exp_spread=20)
    B = I.dd_random(256, 64, 6, exp_spread=20)
    prods = (A[0][:, :, None] * B[0][None, :, :]).reshape(64, -1)
    acc = np.cumsum(prods, axis=1)
    s, e_int, e_fp = _run(acc[:, :-1].ravel(), prods[:, 1:].ravel())
    assert np.array_equal(_bits(e_int), _bits(e_fp))
    # and the error is exact: s + e == a + b in higher precision on a sample
    from fractions import Fraction
    a, b = acc[:, :-1].ravel()[:500], prods[:, 1:].ravel()[:500]
    for x, y, ss, ee in zip(a, b, s[:500], e_int[:500]):
        assert Fraction(float(x)) + Fraction(float(y)) == Fraction(float(ss)) + Fraction(float(ee))


def _run_prod(a, b):
    import ctypes
    import torch
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = torch.empty(3 * len(a), dtype=torch.float64, device="cuda")
    ad, bd = dev(a), dev(b)
    rc = mpg.lib().mpgemm_selftest_two_prod(len(a), ctypes.c_void_p(ad.data_ptr()), ctypes.c_void_p(bd.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 0
    o = out.cpu().numpy().reshape(3, -1)
    return o[0], o[1], o[2]


def _check_prod(a, b):
    """p == the host's IEEE product (both NaN where it is NaN) and the
    integer-pipe error == fma(a, b, -p), bit for bit."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    p, e_int, e_fma = _run_prod(a, b)
    with np.errstate(all="ignore"):
        want = a * b
    nan = np.isnan(want)
    assert np.array_equal(np.isnan(p), nan)
    assert np.array_equal(_bits(p[~nan]), _bits(want[~nan]))
    assert np.array_equal(_bits(e_int), _bits(e_fma))
    return p, e_int


def test_product_error_random_pairs():
    # the DD kernel's product error term on the integer pipe == fma(a, b, -p)
    rng = np.random.default_rng(77)
    n = 1 << 20
    bits = rng.integers(0, 2**63, size=(2, n), dtype=np.uint64) | (rng.integers(0, 2, size=(2, n), dtype=np.uint64) << np.uint64(63))
    a, b = bits[0].view(np.float64), bits[1].view(np.float64)
    _check_prod(a, b)
    # products near 1 (all carries and roundings of the mantissa product)
    a = rng.uniform(1, 2, n) * rng.choice([-1.0, 1.0], n) * np.ldexp(1.0, rng.integers(-500, 500, n))
    b = rng.uniform(1, 2, n) * rng.choice([-1.0, 1.0], n) * np.ldexp(1.0, rng.integers(-500, 500, n))
    _check_prod(a, b)
    # products at the edges of the normal range (overflow, underflow into
    # subnormals and below, subnormal errors)
    a = rng.uniform(1, 2, n) * np.ldexp(1.0, rng.integers(-1022, 1024, n))
    b = rng.uniform(1, 2, n) * np.ldexp(1.0, rng.integers(-1022, 1024, n))
    near = np.abs(np.log2(np.abs(a)) + np.log2(np.abs(b)))
    assert (near > 1000).sum() > 1000
    _check_prod(a, b)


def test_product_roundings():
    # mantissa products one unit either side of a binade (x y just below
    # 2^105 or 2^106: many round up into the next binade, a carry into the
    # exponent field) and exact ties at both product widths, rounding up and
    # down to even
    rng = np.random.default_rng(78)
    xs, ys = [], []
    for _ in range(20000):
        x = int(rng.integers(1 << 52, 1 << 53))
        for top in (106, 105):
            y = ((1 << top) - 1) // x
            if (1 << 52) <= y < (1 << 53):
                xs.append(x); ys.append(y)
    ties = [(3 << 51, (1 << 52) + k) for k in range(1, 400, 2)]                  # P < 2^105
    ties += [(7 << 50, (5 << 50) + 4 + 8 * j) for j in range(200)]               # P >= 2^105
    for x, y in ties:
        P = x * y
        sh = 53 if P >> 105 else 52
        assert P % (1 << sh) == 1 << (sh - 1)                                       # an exact tie
    xs += [x for x, _ in ties]
    ys += [y for _, y in ties]
    a = np.array([np.ldexp(float(v), -52) for v in xs]) * rng.choice([-1.0, 1.0], len(xs))
    b = np.array([np.ldexp(float(v), -52) for v in ys]) * rng.choice([-1.0, 1.0], len(ys))
    p, e = _check_prod(a, b)
    assert ((np.abs(p) == 2.0) | (np.abs(p) == 4.0)).sum() > 100   # roundings into the next binade


def test_product_error_crafted_pairs():
    tiny = np.ldexp(1.0, -1074)
    big = np.finfo(np.float64).max
    u = 2.0 ** -53
    vals = [0.0, -0.0, 1.0, 1.0 + 2 * u, 1.0 - u, 2.0 - 2 * u, np.sqrt(2.0), 3.0, tiny, np.ldexp(1.0, -1022),
            np.ldexp(1.0, -600), np.ldexp(1.0, -511), np.ldexp(1.5, -512), big, np.ldexp(1.0, 600),
            np.ldexp(1.0, 512), np.inf, np.nan, 1.0 / 3.0, np.ldexp(1.0 - u, 1), 1e-300, 1e300]
    vals = np.array(vals + [-v for v in vals])
    a, b = np.meshgrid(vals, vals, indexing="ij")
    _check_prod(a.ravel(), b.ravel())

