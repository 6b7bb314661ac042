"""The DD multiply-accumulate computes TwoProd and TwoSum's error term on
the integer pipe, handing its rare cases (zero, subnormal, infinite or NaN
values, products or errors outside the integer forms' range) to FP64.  Its
step must equal, bit for bit, the same steps with every error term from
FP64 operations (mpgemm_selftest_dd_mac), on random accumulator / operand
pairs, accumulators near the product (cancellations, carries, far above and
below) and every combination of special values; and the block GEMMs must
equal the simple algorithm's result bit for bit (both keep Eq 1's order: k
ascending, the accumulator renormalised every 8 steps; l a multiple of the
16-deep panels so that the block kernels add no padding steps) on random
inputs and on inputs that take the rare cases: zero rows, columns and
entries (+0 and -0), subnormals, products at the ends of the integer
TwoProd's range (2^-917 and 2^1023), accumulators that cancel to zero
exactly, sums that overflow, infinities and NaN (NaN compared as NaN)."""

import numpy as np
import pytest

from gpu_util import dev, host
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")

SHAPES = [(45, 96, 37), (70, 208, 33)]


def _bits(C):
    """The doubles' bits, every NaN mapped to one pattern (the sign and
    payload of a NaN are not specified: a kernel may fold a negation into an
    FMA or not)."""
    b = np.ascontiguousarray(C).view(np.uint64).copy()
    b[np.isnan(C)] = 0x7FF8000000000000
    return b


def _same_as_simple(A, B):
    Ad, Bd = dev(A), dev(B)
    Cs = host(mpg.gemm_dd(Ad, Bd, algo="simple"))
    for n_min in (16, 32):
        Cb = host(mpg.gemm_dd(Ad, Bd, algo="block", n_min=n_min))
        assert np.array_equal(_bits(Cb), _bits(Cs)), n_min
    return Cs


@pytest.mark.parametrize("m,l,n", SHAPES)
def test_random_inputs(m, l, n):
    A, B = I.dd_random(m, l, 301, 20), I.dd_random(l, n, 302, 20)
    _same_as_simple(A, B)


@pytest.mark.parametrize("m,l,n", SHAPES)
def test_zeros(m, l, n):
    rng = np.random.default_rng(303)
    A, B = I.dd_random(m, l, 304, 20), I.dd_random(l, n, 305, 20)
    A[:, 3, :] = 0.0                       # a zero row of A
    B[:, :, 5] = -0.0                      # a zero column of B
    zA = rng.random((m, l)) < 0.1
    A[0][zA] = rng.choice([0.0, -0.0], size=int(zA.sum()))
    A[1][zA] = 0.0
    B[:, 7, :] = 0.0                       # a zero row of B (every product of step 7 is zero)
    _same_as_simple(A, B)


@pytest.mark.parametrize("m,l,n", SHAPES)
def test_subnormals_and_range_ends(m, l, n):
    rng = np.random.default_rng(306)
    A, B = I.dd_random(m, l, 307, 20), I.dd_random(l, n, 308, 20)
    sub = rng.random((m, l)) < 0.05
    A[0][sub] = np.ldexp(rng.uniform(0.5, 1, int(sub.sum())), -1060)        # subnormal
    A[1][sub] = 0.0
    # products at the ends of the integer TwoProd's range: exponent fields
    # summing to 1129 (from 2^-917, inside), 1128 (outside), 3067 (below
    # 2^1023, inside)
    u = lambda k: rng.uniform(1, 2, k) * rng.choice([-1.0, 1.0], k)
    for row, ea, col, eb, ks in ((10, -459, 7, -458, slice(4, 8)), (11, -460, 7, -458, slice(4, 8)),
                                 (12, 511, 6, 510, slice(0, 4))):
        A[0][row, ks] = np.ldexp(u(4), ea)
        A[1][row, ks] = 0.0
        B[0][ks, col] = np.ldexp(u(4), eb)
        B[1][ks, col] = 0.0
    _same_as_simple(A, B)


@pytest.mark.parametrize("m,l,n", SHAPES)
def test_exact_cancellation(m, l, n):
    # small integers against +-1: the accumulator returns to exactly zero
    # many times (sums s = x - x = +0), then grows again
    rng = np.random.default_rng(309)
    A = np.zeros((2, m, l))
    A[0] = rng.integers(1, 4, size=(m, l)).astype(np.float64)
    A[0][:, 1::2] = A[0][:, 0::2]
    B = np.zeros((2, l, n))
    B[0] = 1.0
    B[0][1::2, :] = -1.0
    B[0][:, 0] = rng.choice([-1.0, 1.0], size=l)       # one column that does not cancel
    B[1][:, 1] = 2.0 ** -60                            # one column with nonzero low parts
    C = _same_as_simple(A, B)
    assert np.all(C[0][:, 2:] == 0)


def test_overflow_infinities_nan():
    m, l, n = SHAPES[0]
    A, B = I.dd_random(m, l, 310, 20), I.dd_random(l, n, 311, 20)
    with np.errstate(over="ignore"):
        A[:, 2, :] = np.ldexp(np.abs(A[:, 2, :]), 1022)    # sums of products near 2^1023 overflow
    B[:, :, 3] = np.ldexp(np.abs(B[:, :, 3]), 1)
    A[0, 5, 9] = np.inf
    A[1, 5, 9] = 0.0
    B[0, 20, 4] = np.nan
    B[1, 20, 4] = 0.0
    A[0, 6, 30] = -np.inf
    A[1, 6, 30] = 0.0
    C = _same_as_simple(A, B)
    assert np.isinf(C[0][2, 3]) or np.isnan(C[0][2, 3])
    assert np.all(np.isnan(C[0][:, 4]))


def _run_mac(s, t, ah, al, bh, bl):
    import ctypes
    import torch
    v = np.ascontiguousarray(np.stack([np.asarray(x, dtype=np.float64) for x in (s, t, ah, al, bh, bl)]))
    count = v.shape[1]
    out = torch.empty(8 * count, dtype=torch.float64, device="cuda")
    vd = dev(v)
    rc = mpg.lib().mpgemm_selftest_dd_mac(count, ctypes.c_void_p(vd.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                          None)
    assert rc == 0
    return _bits(out.cpu().numpy().reshape(8, count))


def _check_mac(*planes):
    o = _run_mac(*planes)
    assert np.array_equal(o[0:2], o[2:4])      # the MAC step, bit for bit
    assert np.array_equal(o[4:6], o[6:8])      # and a renormalisation after it


def test_mac_step_equals_fp64_form():
    rng = np.random.default_rng(312)
    n = 1 << 20
    u = 2.0 ** -53
    ah = rng.uniform(-2, 2, n) * np.ldexp(1.0, rng.integers(-520, 520, n))
    bh = rng.uniform(-2, 2, n) * np.ldexp(1.0, rng.integers(-520, 520, n))
    al, bl = ah * u * rng.uniform(-1, 1, n), bh * u * rng.uniform(-1, 1, n)
    p = ah * bh
    with np.errstate(all="ignore"):
        for s in (rng.uniform(-2, 2, n) * np.ldexp(1.0, rng.integers(-1000, 1000, n)), -p, p, p * 3,
                  p * 2.0 ** 60, p * 2.0 ** -60, p * 2.0 ** 55, np.nextafter(-p, 0), np.zeros(n), -np.zeros(n)):
            t = s * u * rng.uniform(-1, 1, n)
            _check_mac(s, t, ah, al, bh, bl)
        # zeros, subnormals, infinities and NaN among the operands and the accumulator
        special = np.array([0.0, -0.0, 2.0 ** -1074, -(2.0 ** -1060), 2.0 ** -1022, np.inf, -np.inf, np.nan, 1.0,
                            -3.0, 2.0 ** 1000, 2.0 ** -1000, 2.0 ** -459, 2.0 ** 511])
        g = np.array(np.meshgrid(special, special, special, indexing="ij")).reshape(3, -1)
        _check_mac(g[0], g[0] * u, g[1], g[1] * u, g[2], np.zeros_like(g[2]))
        _check_mac(g[0], np.zeros_like(g[0]), g[1], np.zeros_like(g[1]), g[2], g[2] * u)
