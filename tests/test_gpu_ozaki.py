"""Parity of the split-precision DD GEMM (CUDA, through the C ABI) with the
oracle: exponents, int8 digits and int32 level sums bit-identical, the DD
result bit-identical (both round the same exact value once), and at the
full 4096 size |C - C_exact| <= 2^-100 |A||B| on sampled entries."""

import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import dev, host, sample_indices
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _lp(k):
    return (k + 127) // 128 * 128


def _split(X, S, by_col):
    import torch
    rows, cols = X.shape[1], X.shape[2]
    inner = rows if by_col else cols
    outer = cols if by_col else rows
    Xd = dev(X)
    ex = torch.zeros(outer, dtype=torch.int32, device="cuda")
    D = torch.full((S, outer, _lp(inner)), 99, dtype=torch.int8, device="cuda")
    rc = mpg.lib().mpgemm_ozaki_split(1 if by_col else 0, rows, cols, _p(Xd), S, _p(ex), _p(D),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    return host(ex), host(D)


@pytest.mark.parametrize("S", [3, 16, 18])
def test_split_bit_exact(S):
    A, B = I.dd_rowcol_scaled(37, 70, 45, seed=11)
    A[:, 5, :] = 0.0
    A[:, 6, 9] = 0.0
    B[:, :, 7] = 0.0          # an all-zero column: exponent 0
    e, DA = _split(A, S, by_col=False)
    f, DB = _split(B, S, by_col=True)
    assert np.array_equal(e, oracle.ozaki_row_expo(A))
    assert np.array_equal(f, oracle.ozaki_col_expo(B))
    oa = oracle.ozaki_slice(A, e, S, by_col=False)
    ob = oracle.ozaki_slice(B, f, S, by_col=True)
    assert np.array_equal(DA[:, :, :70], oa)
    assert not DA[:, :, 70:].any()                      # K padding is zero
    assert np.array_equal(DB[:, :, :70], ob.transpose(0, 2, 1))
    assert not DB[:, :, 70:].any()


@pytest.mark.parametrize("m,l,n,S", [(37, 70, 45, 5), (130, 200, 129, 16), (256, 128, 256, 8)])
def test_levels_bit_exact(m, l, n, S):
    import torch
    A, B = I.dd_rowcol_scaled(m, l, n, seed=m + n)
    e, DA = _split(A, S, False)
    f, DB = _split(B, S, True)
    Lv = torch.zeros((S, m, n), dtype=torch.int32, device="cuda")
    DAd, DBd = dev(DA), dev(DB)          # keep both alive while the kernel runs
    rc = mpg.lib().mpgemm_ozaki_levels(m, l, n, S, _p(DAd), _p(DBd), _p(Lv),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    L = host(Lv)
    Lo = oracle.ozaki_levels(oracle.ozaki_slice(A, e, S, False), oracle.ozaki_slice(B, f, S, True), S)
    assert np.array_equal(L.astype(np.int64), Lo[2:S + 2])


def _ozaki(A, B, S):
    import torch
    m, l, n = A.shape[1], A.shape[2], B.shape[2]
    Ad, Bd = dev(A), dev(B)
    Cd = torch.empty((2, m, n), dtype=torch.float64, device="cuda")
    rc = mpg.lib().mpgemm_dd_ozaki(m, l, n, _p(Ad), _p(Bd), _p(Cd), S,
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, rc
    return host(Cd)


@pytest.mark.parametrize("S", [8, 16])
def test_ozaki_gemm_bit_exact(S):
    A, B = I.dd_rowcol_scaled(40, 70, 33, seed=S)
    C = _ozaki(A, B, S)
    assert np.array_equal(C, oracle.ozaki_gemm(A, B, S))


def test_ozaki_integers_exact_and_edges():
    a, b = I.int_matrix(20, 30, 1, -100, 100), I.int_matrix(30, 10, 2, -100, 100)
    C = _ozaki(I.ints_to_dd(a), I.ints_to_dd(b), 4)
    assert np.array_equal(C[0], (a @ b).astype(np.float64)) and not C[1].any()
    # empty inner dimension
    C0 = _ozaki(np.zeros((2, 3, 0)), np.zeros((2, 0, 4)), 16)
    assert not C0.any()


@pytest.mark.parametrize("n", [4096])
def test_ozaki_full_size_error_bound(n):
    A, B = I.dd_rowcol_scaled(n, n, n, seed=I.seed_for(3))
    C = _ozaki(A, B, 16)
    ii, jj = sample_indices(n, n, 384, seed=9)
    err, absab = oracle.exact_check(A, B, C, ii, jj)
    assert np.max(err / absab) <= 2.0**-100


def test_ozaki_error_falls_with_slices():
    n = 256
    A, B = I.dd_rowcol_scaled(n, n, n, seed=21)
    ii, jj = sample_indices(n, n, 200, seed=1)
    errs = []
    for S in (10, 13, 16):
        err, absab = oracle.exact_check(A, B, _ozaki(A, B, S), ii, jj)
        errs.append(float(np.max(err / absab)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] <= 2.0**-100
