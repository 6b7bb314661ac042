"""The precision selector's a-priori bounds hold for the results they
describe (no GPU).

For every method that the selector offers, the library's bound
|C - AB| <= beta |A||B| (mpgemm_precision_log2_bound) is checked elementwise
against the oracle's result of the same method, the error and |A||B| taken
from exact accumulation.  The oracle gives the same multi-limb results as the
kernels bit for bit and the same split-precision results bit for bit, so the
bounds are checked here on the arithmetic itself, on inputs whose entries lie
at most `spread` binades below their row (A) or column (B) maximum, with few
slices so that the truncation terms dominate."""

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1710_01839_gb300 import inputs as I

mpg = pytest.importorskip("paper_1710_01839_gb300")


@pytest.fixture(scope="module")
def built():
    try:
        mpg.lib()
    except Exception as e:   # library not built in this checkout
        pytest.skip(str(e))
    return mpg


def _terms(rng, lead, T):
    """T-term non-overlapping expansions led by `lead` (each term below half
    an ulp of the one before)."""
    X = [lead]
    for _ in range(T - 1):
        X.append(X[-1] * 2.0 ** -53 * rng.uniform(-0.5, 0.5, lead.shape) * 2.0 ** -rng.integers(0, 4, lead.shape))
    return np.stack(X)


def _spread_matrix(rng, r, c, spread, by_col, T):
    """Entries sign * U[1/2, 1) * 2^(g - x), g per row (A) or column (B),
    x ~ U{0..spread}: every entry within `spread` binades of its maximum."""
    g = rng.integers(-12, 12, size=(1, c) if by_col else (r, 1))
    x = rng.integers(0, spread + 1, size=(r, c))
    lead = rng.uniform(0.5, 1.0, (r, c)) * rng.choice([-1.0, 1.0], (r, c)) * 2.0 ** (g - x)
    return _terms(rng, lead, T)


def _ratio(A, B, C):
    m, n = A.shape[1], B.shape[2]
    ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    err, absab = oracle.exact_check(A, B, C, ii.ravel(), jj.ravel())
    return np.max(err / absab)


M, L, N = 6, 40, 5


@pytest.mark.parametrize("spread", [0, 3])
@pytest.mark.parametrize("method,S", [("ozaki_int8", 3), ("ozaki_int8", 5), ("ozaki_int8", 8),
                                      ("ozaki_e4m3", 4), ("ozaki_e4m3", 7), ("ozaki_e4m3", 11)])
def test_dd_split_bounds(built, method, S, spread):
    rng = np.random.default_rng(1000 * S + spread)
    A = _spread_matrix(rng, M, L, spread, False, 2)
    B = _spread_matrix(rng, L, N, spread, True, 2)
    C = oracle.ozaki_gemm(A, B, S) if method == "ozaki_int8" else oracle.ozaki_gemm_b32(A, B, S)
    beta = 2.0 ** built.precision_log2_bound(method, L, num_slices=S, spread=spread)
    r = _ratio(A, B, C)
    assert 0 < r <= beta, (r, beta)


@pytest.mark.parametrize("spread", [0, 3])
@pytest.mark.parametrize("S", [10, 24, 36])
def test_qd_split_bounds(built, S, spread):
    rng = np.random.default_rng(500 + S + spread)
    A = _spread_matrix(rng, M, L, spread, False, 4)
    B = _spread_matrix(rng, L, N, spread, True, 4)
    C = oracle.ozaki_gemm_b32_terms(A, B, S)
    lb = built.precision_log2_bound("ozaki_qd", L, num_slices=S, spread=spread)
    assert not np.isnan(lb)
    r = _ratio(A, B, C)
    assert 0 < r <= 2.0 ** lb, (r, 2.0 ** lb)


def test_dd_qd_bounds(built):
    rng = np.random.default_rng(7)
    A2, B2 = _spread_matrix(rng, M, L, 20, False, 2), _spread_matrix(rng, L, N, 20, True, 2)
    assert _ratio(A2, B2, oracle.dd_gemm(A2, B2)) <= 2.0 ** built.precision_log2_bound("dd", L)
    A4, B4 = _spread_matrix(rng, M, L, 20, False, 4), _spread_matrix(rng, L, N, 20, True, 4)
    assert _ratio(A4, B4, oracle.qd_gemm(A4, B4)) <= 2.0 ** built.precision_log2_bound("qd", L)


def _mp_fraction(Y, w, i, j):
    e = int(np.int32(np.uint32(Y[0, i, j])))
    f = int(Y[1, i, j])
    if f & 2:
        return Fraction(0)
    M = sum(int(Y[2 + q, i, j]) << (32 * q) for q in range(w))
    v = Fraction(M) * Fraction(2) ** (e - 32 * w)
    return -v if f & 1 else v


@pytest.mark.parametrize("bits", [64, 128, 256, 512])
def test_multi_limb_bounds(built, bits):
    # full-width random mantissas; the error and |A||B| in exact rationals
    w = bits // 32
    Am, Bm = I.mp_random(M, L, w, 300 + bits), I.mp_random(L, N, w, 400 + bits)
    Cm = oracle.mp_gemm(Am, Bm, bits)
    a = [[_mp_fraction(Am, w, i, k) for k in range(L)] for i in range(M)]
    b = [[_mp_fraction(Bm, w, k, j) for j in range(N)] for k in range(L)]
    worst = Fraction(0)
    for i in range(M):
        for j in range(N):
            exact = sum(a[i][k] * b[k][j] for k in range(L))
            absab = sum(abs(a[i][k] * b[k][j]) for k in range(L))
            worst = max(worst, abs(_mp_fraction(Cm, w, i, j) - exact) / absab)
    lb = built.precision_log2_bound("mp", L, prec_bits=bits)
    assert 0 < worst and math.log2(worst) <= lb, (math.log2(worst), lb)


@pytest.mark.parametrize("method,T,bits", [("dd_via_mp", 2, 128), ("dd_via_mp", 2, 256), ("qd_via_mp", 4, 256),
                                           ("qd_via_mp", 4, 512)])
def test_integer_pipe_bounds(built, method, T, bits):
    rng = np.random.default_rng(T * bits)
    A, B = _spread_matrix(rng, M, L, 20, False, T), _spread_matrix(rng, L, N, 20, True, T)
    C = oracle.gemm_via_mp(A, B, bits)
    assert _ratio(A, B, C) <= 2.0 ** built.precision_log2_bound(method, L, prec_bits=bits)
