"""The split-precision DD GEMM with FP8 (e4m3) digits against the oracle:
balanced base-32 digits bit-identical (decoded from their e4m3 codes), level
sums bit-identical (the f32 tensor-core accumulation is exact because every
partial sum is an integer below 2^24), the DD result bit-identical, and
|C - C_exact| <= 2^-100 |A||B| at the full 4096 size on sampled entries."""

import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import dev, host, sample_indices
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")

E4M3 = 1


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _sp():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _lp(k):
    return (k + 127) // 128 * 128


def decode_e4m3(codes: np.ndarray) -> np.ndarray:
    """Exact values of e4m3 codes that hold small integers (test helper)."""
    c = codes.astype(np.int64)
    sign = np.where(c & 0x80, -1, 1)
    e = (c >> 3) & 0xF
    mant = c & 7
    val = np.where(e == 0, mant / 8.0 * 2.0**-6, (1 + mant / 8.0) * 2.0 ** (e - 7))
    return (sign * val).astype(np.float64)


def _split(X, S, by_col):
    import torch
    rows, cols = X.shape[1], X.shape[2]
    inner = rows if by_col else cols
    outer = cols if by_col else rows
    Xd = dev(X)
    ex = torch.zeros(outer, dtype=torch.int32, device="cuda")
    D = torch.full((S, outer, _lp(inner)), 0x7F, dtype=torch.uint8, device="cuda")
    rc = mpg.lib().mpgemm_ozaki_split_ex(E4M3, 1 if by_col else 0, rows, cols, _p(Xd), S, _p(ex), _p(D), _sp())
    assert rc == 0, rc
    return host(ex), host(D)


# l = 71: odd row length (scalar loads); l = 300: several 256-row blocks per
# column exponent and several 64-row tiles of the transposing column split.
@pytest.mark.parametrize("S", [4, 22, 24])
@pytest.mark.parametrize("m,l,n", [(37, 70, 45), (37, 71, 45), (130, 300, 70)])
def test_fp8_digits_bit_exact(S, m, l, n):
    A, B = I.dd_rowcol_scaled(m, l, n, seed=31 + l)
    A[:, 5, :] = 0.0
    A[:, 6, 9] = 0.0
    B[:, :, 7] = 0.0          # an all-zero column: exponent 0
    B[:, 3, 8] = 0.0
    e, DA = _split(A, S, by_col=False)
    f, DB = _split(B, S, by_col=True)
    assert np.array_equal(e, oracle.ozaki_row_expo(A))
    assert np.array_equal(f, oracle.ozaki_col_expo(B))
    va, vb = decode_e4m3(DA), decode_e4m3(DB)
    assert np.all(va == np.round(va)) and np.abs(va).max() <= 16
    oa = oracle.ozaki_slice_b32(A, e, S, by_col=False)
    ob = oracle.ozaki_slice_b32(B, f, S, by_col=True)
    assert np.array_equal(va[:, :, :l], oa.astype(np.float64))
    assert not va[:, :, l:].any()
    assert np.array_equal(vb[:, :, :l], ob.transpose(0, 2, 1).astype(np.float64))
    assert not vb[:, :, l:].any()


# (512, 16, 1024, 24): 384 tile-level jobs, so every CTA of the persistent
# kernel runs several and cycles both tensor-memory accumulators;
# (130, 4500, 24, 16) and (40, 3300, 30, 22): levels with more pairs than one
# exact f32 chunk holds (Q = 2^16 / lp = 14 and 19), added chunk by chunk.
@pytest.mark.parametrize("m,l,n,S", [(37, 70, 45, 6), (130, 200, 129, 22), (256, 192, 256, 24),
                                     (512, 16, 1024, 24), (130, 4500, 24, 16), (40, 3300, 30, 22)])
def test_fp8_levels_bit_exact(m, l, n, S):
    import torch
    A, B = I.dd_rowcol_scaled(m, l, n, seed=m + n + 1)
    e, DA = _split(A, S, False)
    f, DB = _split(B, S, True)
    Lv = torch.zeros((S, m, n), dtype=torch.int32, device="cuda")
    DAd, DBd = dev(DA), dev(DB)
    rc = mpg.lib().mpgemm_ozaki_levels_ex(E4M3, m, l, n, S, _p(DAd), _p(DBd), _p(Lv), _sp())
    assert rc == 0
    Lo = oracle.ozaki_levels(oracle.ozaki_slice_b32(A, e, S, False), oracle.ozaki_slice_b32(B, f, S, True), S)
    assert np.array_equal(host(Lv).astype(np.int64), Lo[2:S + 2])


def test_fp8_levels_reject_unaligned_digits():
    import torch
    DA = torch.zeros((2, 8, 128), dtype=torch.uint8, device="cuda")
    DB = torch.zeros((2, 8, 128), dtype=torch.uint8, device="cuda")
    Lv = torch.zeros((2, 8, 8), dtype=torch.int32, device="cuda")
    rc = mpg.lib().mpgemm_ozaki_levels_ex(E4M3, 8, 100, 8, 2, ctypes.c_void_p(DA.data_ptr() + 1), _p(DB), _p(Lv),
                                          _sp())
    assert rc == -1


def _ozaki_fp8(A, B, S):
    import torch
    m, l, n = A.shape[1], A.shape[2], B.shape[2]
    Ad, Bd = dev(A), dev(B)
    Cd = torch.empty((2, m, n), dtype=torch.float64, device="cuda")
    rc = mpg.lib().mpgemm_dd_ozaki_ex(m, l, n, _p(Ad), _p(Bd), _p(Cd), S, E4M3, _sp())
    assert rc == 0, rc
    return host(Cd)


@pytest.mark.parametrize("S", [12, 22])
def test_fp8_gemm_bit_exact(S):
    A, B = I.dd_rowcol_scaled(40, 70, 33, seed=S + 50)
    assert np.array_equal(_ozaki_fp8(A, B, S), oracle.ozaki_gemm_b32(A, B, S))


def test_fp8_integers_exact():
    a, b = I.int_matrix(20, 30, 3, -100, 100), I.int_matrix(30, 10, 4, -100, 100)
    C = _ozaki_fp8(I.ints_to_dd(a), I.ints_to_dd(b), 6)
    assert np.array_equal(C[0], (a @ b).astype(np.float64)) and not C[1].any()


def test_fp8_full_size_error_bound():
    n = 4096
    A, B = I.dd_rowcol_scaled(n, n, n, seed=I.seed_for(3))
    C = _ozaki_fp8(A, B, 22)
    ii, jj = sample_indices(n, n, 384, seed=11)
    err, absab = oracle.exact_check(A, B, C, ii, jj)
    assert np.max(err / absab) <= 2.0**-100


def test_fp8_rejects_too_long_inner_dimension():
    L = mpg.lib()
    assert L.mpgemm_dd_ozaki_ex(4, 70000, 4, ctypes.c_void_p(16), ctypes.c_void_p(16), ctypes.c_void_p(16), 22,
                                E4M3, None) == -2
    assert L.mpgemm_dd_ozaki_ex(4, 4, 4, None, None, None, 25, E4M3, None) == -1


def test_fp8_maximum_inner_dimension_and_degenerate_shapes():
    """l = 65536, the largest inner dimension whose slice-pair sums stay
    exact in f32 (Q = 1: every pair is its own chunk, added chunk by chunk),
    and 1 x 1 x 1 / 1 x l x 1 products."""
    A, B = I.dd_rowcol_scaled(3, 65536, 2, seed=71)
    assert np.array_equal(_ozaki_fp8(A, B, 8), oracle.ozaki_gemm_b32(A, B, 8))
    for (m, l, n) in [(1, 1, 1), (1, 300, 1), (2, 1, 3)]:
        A, B = I.dd_rowcol_scaled(m, l, n, seed=72 + l)
        assert np.array_equal(_ozaki_fp8(A, B, 22), oracle.ozaki_gemm_b32(A, B, 22))
