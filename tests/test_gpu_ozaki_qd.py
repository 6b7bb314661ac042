"""The split-precision QD GEMM (FP8 digits of 4-term expansions) against the
oracle: exponents and digits bit-identical, the QD result bit-identical
(both round the same exact value greedily to four doubles), integer products
exact, and at 1024^3 |C - C_exact| <= 4 l 2^-208 |A||B| on sampled entries."""

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


def _sp():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _decode_e4m3(codes):
    c = codes.astype(np.int64)
    sign = np.where(c & 0x80, -1, 1)
    e = (c >> 3) & 0xF
    mant = c & 7
    val = np.where(e == 0, mant / 8.0 * 2.0**-6, (1 + mant / 8.0) * 2.0 ** (e - 7))
    return (sign * val).astype(np.int64)


def _split(X, S, by_col):
    import torch
    rows, cols = X.shape[1], X.shape[2]
    inner, outer = (rows, cols) if by_col else (cols, rows)
    lp = (inner + 127) // 128 * 128
    Xd = dev(X)
    ex = torch.zeros(outer, dtype=torch.int32, device="cuda")
    D = torch.full((S, outer, lp), 0x7F, dtype=torch.uint8, device="cuda")
    assert mpg.lib().mpgemm_ozaki_split_terms(4, 1 if by_col else 0, rows, cols, _p(Xd), S, _p(ex), _p(D), _sp()) == 0
    return host(ex), _decode_e4m3(host(D))


@pytest.mark.parametrize("S", [10, 44, 48])
@pytest.mark.parametrize("m,l,n", [(37, 70, 45), (20, 301, 70)])
def test_qd_digits_bit_exact(S, m, l, n):
    A, B = I.qd_rowcol_scaled(m, l, n, seed=61 + l)
    A[:, 3, :] = 0.0
    A[2:, 5, :] = 0.0                     # DD-like entries
    B[:, :, 6] = 0.0                      # an all-zero column: exponent 0
    e, DA = _split(A, S, by_col=False)
    f, DB = _split(B, S, by_col=True)
    assert np.array_equal(e, oracle.ozaki_row_expo(A))
    assert np.array_equal(f, oracle.ozaki_col_expo(B))
    assert np.array_equal(DA[:, :, :l], oracle.ozaki_slice_b32_terms(A, e, S, False))
    assert not DA[:, :, l:].any()
    assert np.array_equal(DB[:, :, :l], oracle.ozaki_slice_b32_terms(B, f, S, True).transpose(0, 2, 1))
    assert not DB[:, :, l:].any()


@pytest.mark.parametrize("m,l,n,S", [(40, 70, 33, 44), (130, 300, 129, 48), (64, 40, 96, 12)])
def test_qd_split_gemm_bit_exact(m, l, n, S):
    A, B = I.qd_rowcol_scaled(m, l, n, seed=m + n + S)
    C = host(mpg.gemm_split(dev(A), dev(B), slices=S))
    assert np.array_equal(C, oracle.ozaki_gemm_b32_terms(A, B, S))


def test_qd_split_integers_exact():
    a, b = I.int_matrix(24, 33, 7, -1000, 1000), I.int_matrix(33, 19, 8, -1000, 1000)
    C = host(mpg.gemm_split(dev(I.ints_to_qd(a)), dev(I.ints_to_qd(b)), slices=10))
    assert np.array_equal(C[0], (a @ b).astype(np.float64)) and not C[1:].any()


def test_qd_split_full_size_bound():
    n = 1024
    A, B = I.qd_rowcol_scaled(n, n, n, seed=I.seed_for(1, 44))
    C = host(mpg.gemm_split(dev(A), dev(B)))           # default S = 44
    ii, jj = sample_indices(n, n, 256, seed=44)
    err, absab = oracle.exact_check(A, B, C, ii, jj)
    assert np.max(err / absab) <= 4 * n * 2.0**-208


def test_qd_split_arguments():
    L = mpg.lib()
    assert L.mpgemm_qd_ozaki(4, 4, 4, None, None, None, 49, None) == -1
    assert L.mpgemm_qd_ozaki(4, 70000, 4, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), 44,
                             None) == -2
    assert L.mpgemm_qd_ozaki_slices_default() == 44
    assert L.mpgemm_ozaki_split_terms(2, 0, 4, 4, ctypes.c_void_p(16), 10, ctypes.c_void_p(16),
                                      ctypes.c_void_p(16), None) == -2


def test_qd_split_bound_on_the_qd_workload():
    """The large QD workload (per-element exponents 2^U{-20..20}, as the plain
    QD kernels are benchmarked) at 1024^3 with the default 44 slices."""
    n = 1024
    A = I.qd_random(n, n, I.seed_for(1, 0), exp_spread=20)
    B = I.qd_random(n, n, I.seed_for(1, 1), exp_spread=20)
    C = host(mpg.gemm_split(dev(A), dev(B)))
    ii, jj = sample_indices(n, n, 256, seed=45)
    err, absab = oracle.exact_check(A, B, C, ii, jj)
    assert np.max(err / absab) <= 4 * n * 2.0**-208


def test_qd_split_maximum_inner_dimension_and_degenerate_shapes():
    A, B = I.qd_rowcol_scaled(2, 65536, 2, seed=73)
    C = host(mpg.gemm_split(dev(A), dev(B), slices=6))
    assert np.array_equal(C, oracle.ozaki_gemm_b32_terms(A, B, 6))
    for (m, l, n) in [(1, 1, 1), (1, 130, 1), (3, 1, 2)]:
        A, B = I.qd_rowcol_scaled(m, l, n, seed=74 + l)
        C = host(mpg.gemm_split(dev(A), dev(B), slices=44))
        assert np.array_equal(C, oracle.ozaki_gemm_b32_terms(A, B, 44))
    import torch
    Z = torch.zeros((4, 3, 0), dtype=torch.float64, device="cuda")
    Z2 = torch.zeros((4, 0, 5), dtype=torch.float64, device="cuda")
    assert not host(mpg.gemm_split(Z, Z2)).any()              # empty inner dimension: C = 0
