"""The Strassen operand and assembly passes (Eq 3's sums and differences,
each rounded in DD) compute the accurate double-word addition with three of
its four error terms on the integer pipe and recompute, with the FP64 error
terms, every element whose operands the integer form flags as rare
(infinite, NaN or subnormal values, the last Fast2Sum's operands out of
exponent order).  Checked
here through mpgemm_selftest_dd_add:
  - unflagged results equal the FP64 form bit for bit, on the benchmark's
    operand pairs (none flagged there), near cancellations of the high
    parts, exact cancellations, zeros of both signs, and every combination
    of special values;
  - every operand set with an infinity or a NaN is flagged;
  - the passes' result (the FP64 form where flagged) equals the oracle's
    double-word addition (Knuth's TwoSum, then the same Fast2Sum steps) as
    values (the two TwoSums may give zeros of opposite sign);
and at the GEMM level, DD Strassen on inputs that take the flagged path
(subnormal entries, near-cancelling quadrants) stays within its bound."""

import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import dev, host, sample_indices
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")


def _run(xh, xl, yh, yl):
    import torch
    v = np.ascontiguousarray(np.stack([xh, xl, yh, yl]).astype(np.float64).reshape(4, -1))
    n = v.shape[1]
    out = torch.empty(5 * n, dtype=torch.float64, device="cuda")
    vd = dev(v)
    rc = mpg.lib().mpgemm_selftest_dd_add(n, ctypes.c_void_p(vd.data_ptr()), ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 0
    o = out.cpu().numpy().reshape(5, n)
    return o[0:2], o[2:4], o[4] != 0.0


def _bits(x):
    return np.ascontiguousarray(x).view(np.uint64)


def _check_unflagged_equal(z_int, z_fp, rare):
    keep = ~rare
    assert np.array_equal(_bits(z_int[:, keep]), _bits(z_fp[:, keep]))


def _dd_pairs(n, seed, spread=20):
    X = I.dd_random(1, n, seed, spread).reshape(2, n)
    Y = I.dd_random(1, n, seed + 1, spread).reshape(2, n)
    return X, Y


def test_benchmark_pairs_none_flagged():
    X, Y = _dd_pairs(1 << 20, 41)
    for sgn in (1.0, -1.0):                         # sums and differences
        z_int, z_fp, rare = _run(X[0], X[1], sgn * Y[0], sgn * Y[1])
        assert not rare.any()
        assert np.array_equal(_bits(z_int), _bits(z_fp))


@pytest.mark.parametrize("ulps", [0, 1, 2, 40])
def test_near_cancellation_of_the_high_parts(ulps):
    # y's high part within a few ulps of -x's: the sum is of the order of
    # the low parts, the Fast2Sum operands may come out of exponent order
    rng = np.random.default_rng(50 + ulps)
    n = 1 << 18
    X, _ = _dd_pairs(n, 43)
    yh = -np.nextafter(X[0], X[0] * 2) if ulps == 1 else -X[0]
    if ulps > 1:
        k = rng.integers(-ulps, ulps + 1, n)
        yh = -(X[0] + k * np.spacing(X[0]))
    yl = -X[1] * rng.uniform(0.25, 4, n) * rng.choice([-1.0, 1.0], n)
    z_int, z_fp, rare = _run(X[0], X[1], yh, yl)
    _check_unflagged_equal(z_int, z_fp, rare)


def test_exact_cancellations_and_signed_zeros():
    X, _ = _dd_pairs(4096, 44)
    z = np.zeros(4096)
    cases = [
        (X[0], X[1], -X[0], -X[1]),                  # x + (-x) = 0
        (X[0], z, -X[0], z),
        (X[0], -z, -X[0], -z),
        (z, z, z, z), (-z, -z, -z, -z), (z, -z, -z, z),
        (X[0], X[1], z, z), (z, z, X[0], X[1]),       # x + 0
        (X[0], z, X[0], z),                           # lo parts zero
    ]
    for c in cases:
        z_int, z_fp, rare = _run(*c)
        assert not rare.any()
        assert np.array_equal(_bits(z_int), _bits(z_fp))


def test_special_values_every_combination():
    tiny = np.ldexp(1.0, -1074)
    big = np.finfo(np.float64).max
    u = 2.0 ** -53
    vals = [0.0, -0.0, 1.0, -1.0, 1.0 + 2 * u, 1.0 - u, 3.0, u, u * u, tiny, 2 * tiny, np.ldexp(1.0, -1022),
            np.ldexp(1.0, -1022) * (1 - 2 * u), big, -big, np.inf, -np.inf, np.nan, np.ldexp(1.0, 1023),
            np.ldexp(1.0, -1000), 1e300]
    vals = np.array(vals + [-v for v in vals[2:]])
    g = np.meshgrid(vals, vals, vals, vals, indexing="ij")
    xh, xl, yh, yl = (a.ravel() for a in g)
    z_int, z_fp, rare = _run(xh, xl, yh, yl)
    _check_unflagged_equal(z_int, z_fp, rare)
    nonfinite = ~np.isfinite(xh) | ~np.isfinite(xl) | ~np.isfinite(yh) | ~np.isfinite(yl)
    assert rare[nonfinite].all()
    assert (~rare).sum() > len(rare) // 10


def test_against_the_oracle_double_word_addition():
    rng = np.random.default_rng(47)
    n = 6000
    X, Y = _dd_pairs(n, 45, spread=60)
    Y[:, : n // 3] = -X[:, : n // 3] * (1 + rng.integers(-3, 4, n // 3) * 2.0 ** -52)   # near cancellations
    Y[1, n // 3: n // 2] = 0.0
    z_int, z_fp, rare = _run(X[0], X[1], Y[0], Y[1])
    z = np.where(rare, z_fp, z_int)                  # what the passes store
    want = np.array([oracle.dd_add(X[:, i], Y[:, i]) for i in range(n)]).T
    assert np.array_equal(z, want)                   # as values: +0 == -0


@pytest.mark.parametrize("depth", [1, 3])
def test_strassen_with_subnormal_entries_within_bound(depth):
    n = 128
    A, B = I.dd_random(n, n, 760 + depth), I.dd_random(n, n, 770 + depth)
    rng = np.random.default_rng(depth)
    pick = rng.random((n, n)) < 0.05
    A[0][pick] = np.ldexp(rng.uniform(1, 2, int(pick.sum())), -1060)   # subnormal entries, low parts zero
    A[1][pick] = 0.0
    C = host(mpg.gemm_dd(dev(A), dev(B), algo="strassen", n_min=16, depth=depth))
    ii, jj = sample_indices(n, n, 600, seed=depth)
    err, _ = oracle.exact_check(A, B, C, ii, jj)
    amax = np.max(np.abs(A[0] + A[1]))
    bmax = np.max(np.abs(B[0] + B[1]))
    assert np.max(err) <= 2.0**-96 * n * amax * bmax


@pytest.mark.parametrize("depth", [1, 2, 4])
def test_strassen_with_cancelling_quadrants_within_bound(depth):
    # A22 = -A11 + tiny and B22 = -B11 + tiny: the first level's P1
    # operands (A11 + A22, B11 + B22) cancel in their high parts
    n = 256
    A, B = I.dd_random(n, n, 780 + depth), I.dd_random(n, n, 790 + depth)
    h = n // 2
    for X, s in ((A, 11), (B, 12)):
        rng = np.random.default_rng(s)
        X[0, h:, h:] = -X[0, :h, :h] * (1 + rng.integers(-2, 3, (h, h)) * 2.0 ** -52)
        X[1, h:, h:] = -X[1, :h, :h] * rng.uniform(0.5, 2, (h, h))
    C = host(mpg.gemm_dd(dev(A), dev(B), algo="strassen", n_min=16, depth=depth))
    ii, jj = sample_indices(n, n, 600, seed=depth)
    err, _ = oracle.exact_check(A, B, C, ii, jj)
    amax = np.max(np.abs(A[0] + A[1]))
    bmax = np.max(np.abs(B[0] + B[1]))
    assert np.max(err) <= 2.0**-96 * n * amax * bmax
