"""Parity of the DD / QD GEMM on the integer pipe (mpgemm_dd_via_mp,
mpgemm_qd_via_mp, and the conversions mpgemm_terms_to_mp /
mpgemm_mp_to_terms) with the oracle.

Bars: the conversions and the GEMMs are bit-identical to the oracle's
(conversion, multi-limb GEMM, conversion) at the same precision, algorithm,
n_min and depth; at the bench's full sizes sampled entries are within the
DD / QD bounds of the exact product (and far inside them).
"""

import numpy as np
import pytest
import oracle
from gpu_util import DD_BOUND, QD_BOUND, bound_ratio, dev, host, sample_indices
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")


@pytest.mark.parametrize("T,bits", [(2, 64), (2, 128), (2, 256), (4, 256), (4, 512)])
def test_conversions_bit_exact(T, bits):
    gen = I.dd_random if T == 2 else I.qd_random
    X = gen(37, 29, 500 + bits, exp_spread=20)
    X[T - 1, :5] *= 2.0 ** -90          # expansions wider than p bits: rounding
    X[:, 5, :3] = 0.0
    X[1, 6, :2] = -0.0
    Y = host(mpg.to_mp(dev(X), bits), mp=True)
    assert np.array_equal(Y, oracle.terms_to_mp(X, bits))
    w = bits // 32
    Z = I.mp_random(31, 23, w, 600 + bits, emin=-300, emax=300)
    Z[2:, 0, :4] = 0
    Z[2 + w - 1, 0, :4] = 0x80000000
    Z[2:2 + w - 1, 1, :4] = 0xFFFFFFFF
    Xo = mpg.from_mp(dev(Z), bits, T).cpu().numpy()
    assert np.array_equal(Xo.view(np.uint64), oracle.mp_to_terms(Z, bits, T).view(np.uint64))
    assert mpg.stream_status() == 0


@pytest.mark.parametrize("algo,n_min,depth", [("simple", 16, 0), ("block", 16, 0), ("block", 64, 0),
                                              ("strassen", 16, 1), ("strassen", 16, 2)])
def test_dd_via_mp_bit_exact(algo, n_min, depth):
    m, l, n = 45, 37, 29
    A = I.dd_random(m, l, 700, exp_spread=20)
    B = I.dd_random(l, n, 701, exp_spread=20)
    C = mpg.gemm_via_mp(dev(A), dev(B), 128, algo=algo, n_min=n_min, depth=depth).cpu().numpy()
    Co = oracle.gemm_via_mp(A, B, 128, algo=algo, n_min=n_min, depth=depth)
    assert np.array_equal(C.view(np.uint64), Co.view(np.uint64))
    assert mpg.stream_status() == 0


@pytest.mark.parametrize("algo,depth", [("block", 0), ("strassen", 2)])
@pytest.mark.parametrize("bits", [256, 512])
def test_qd_via_mp_bit_exact(algo, depth, bits):
    m, l, n = 26, 33, 21
    A = I.qd_random(m, l, 710, exp_spread=20)
    B = I.qd_random(l, n, 711, exp_spread=20)
    C = mpg.gemm_via_mp(dev(A), dev(B), bits, algo=algo, n_min=16, depth=depth).cpu().numpy()
    Co = oracle.gemm_via_mp(A, B, bits, algo=algo, n_min=16, depth=depth)
    assert np.array_equal(C.view(np.uint64), Co.view(np.uint64))
    assert mpg.stream_status() == 0


def test_dd_via_mp_full_size_rows_bit_exact():
    # the bench's DD 2048^3 inputs through the block algorithm: three full
    # rows of C bit-identical to the oracle's conversion + multi-limb rows
    n, bits = 2048, 128
    A = I.dd_random(n, n, I.seed_for(1, 0), exp_spread=20)
    B = I.dd_random(n, n, I.seed_for(1, 1), exp_spread=20)
    C = mpg.gemm_via_mp(dev(A), dev(B), bits, algo="block", n_min=16).cpu().numpy()
    Am, Bm = oracle.terms_to_mp(A, bits), oracle.terms_to_mp(B, bits)
    for r0 in (0, 1023, n - 1):
        Cm = oracle.mp_gemm(Am, Bm, prec_bits=bits, algo="block", n_min=16, rows=(r0, r0 + 1))
        Co = oracle.mp_to_terms(np.ascontiguousarray(Cm[:, r0:r0 + 1]), bits, 2)
        assert np.array_equal(C[:, r0:r0 + 1].view(np.uint64), Co.view(np.uint64)), r0
    assert mpg.stream_status() == 0


def _within_limb_bound(A, B, C, ii, jj, p, last):
    """|c - c_exact| <= 2^-last |c| (the final rounding to T doubles) +
    (2 l + 4) 2^-p sum|a||b| (p-bit conversions and arithmetic)."""
    l = A.shape[2]
    err, absab = oracle.exact_check(A, B, C, ii, jj)
    cabs = np.abs(C[0][ii, jj])
    return bool(np.all(err <= 2.0 ** -last * cabs + (2 * l + 4) * 2.0 ** -p * absab))


def test_dd_via_mp_full_size_within_bound():
    # the bench's DD 2048^3 workload, Strassen depth 3: sampled entries of C
    # within the DD bound of the exact product, and within the 128-bit bound
    # (the final rounding to two doubles dominates)
    n = 2048
    A = I.dd_random(n, n, I.seed_for(1, 0), exp_spread=20)
    B = I.dd_random(n, n, I.seed_for(1, 1), exp_spread=20)
    C = mpg.gemm_via_mp(dev(A), dev(B), 128, algo="strassen", n_min=512, depth=3).cpu().numpy()
    ii, jj = sample_indices(n, n, 64, seed=3)
    assert bound_ratio(A, B, C, ii, jj, DD_BOUND) <= 2.0 ** -14
    assert _within_limb_bound(A, B, C, ii, jj, 128, 105)
    assert mpg.stream_status() == 0


def test_qd_via_mp_full_size_within_bound():
    n = 1024
    A = I.qd_random(n, n, I.seed_for(1, 0), exp_spread=20)
    B = I.qd_random(n, n, I.seed_for(1, 1), exp_spread=20)
    C = mpg.gemm_via_mp(dev(A), dev(B), 256, algo="strassen", n_min=512, depth=3).cpu().numpy()
    ii, jj = sample_indices(n, n, 32, seed=4)
    assert bound_ratio(A, B, C, ii, jj, QD_BOUND) <= 2.0 ** -14
    assert _within_limb_bound(A, B, C, ii, jj, 256, 210)
    assert mpg.stream_status() == 0


def test_via_mp_empty_and_degenerate():
    A = dev(I.dd_random(5, 0, 1))
    B = dev(I.dd_random(0, 4, 2))
    C = mpg.gemm_via_mp(A, B, 128)
    assert C.shape == (2, 5, 4) and not C.cpu().numpy().any()
    A = dev(I.dd_random(0, 3, 1))
    B = dev(I.dd_random(3, 4, 2))
    assert mpg.gemm_via_mp(A, B, 128).shape == (2, 0, 4)
    # a 1 x 1 x 1 product and an all-zero row
    A = I.dd_random(3, 1, 3)
    A[:, 1] = 0.0
    B = I.dd_random(1, 1, 4)
    C = mpg.gemm_via_mp(dev(A), dev(B), 128).cpu().numpy()
    assert np.array_equal(C.view(np.uint64), oracle.gemm_via_mp(A, B, 128).view(np.uint64))
    assert mpg.stream_status() == 0


def test_via_mp_rejects_bad_precision_and_flags_nonfinite():
    A = dev(I.dd_random(4, 4, 1))
    B = dev(I.dd_random(4, 4, 2))
    for bits in (96, 2048, 40):
        with pytest.raises(mpg.MpgemmError):
            mpg.gemm_via_mp(A, B, bits)
    A2 = A.clone()
    A2[0, 1, 2] = float("inf")
    mpg.gemm_via_mp(A2, B, 128)
    assert mpg.stream_status() == -1     # MPGEMM_EINVAL: an input was not finite
    assert mpg.stream_status() == 0      # read and cleared


def test_via_mp_results_outside_the_double_range_are_flagged():
    # 2^600 x 2^600 overflows a double; 2^-500 (1 + 2^-50) squared leaves a
    # second DD term near 2^-1100, below the normal range: both are written
    # as zero and reported as MPGEMM_EOVERFLOW, without a fault
    big = np.zeros((2, 1, 1))
    big[0] = 2.0 ** 600
    C = mpg.gemm_via_mp(dev(big), dev(big), 128).cpu().numpy()
    assert not C.any()
    assert mpg.stream_status() == -4
    small = np.zeros((2, 1, 1))
    small[0] = 2.0 ** -500 * (1 + 2.0 ** -50)
    C = mpg.gemm_via_mp(dev(small), dev(small), 128).cpu().numpy()
    assert C[0, 0, 0] == 2.0 ** -1000 * (1 + 2.0 ** -49) and C[1, 0, 0] == 0.0
    assert mpg.stream_status() == -4
    # in range again: no flag
    ok = np.zeros((2, 1, 1))
    ok[0] = 3.0
    C = mpg.gemm_via_mp(dev(ok), dev(ok), 128).cpu().numpy()
    assert C[0, 0, 0] == 9.0 and C[1, 0, 0] == 0.0
    assert mpg.stream_status() == 0


def test_via_mp_caller_workspace_and_partition():
    # the conversions' copies and Strassen's workspace from one caller
    # buffer of exactly mpgemm_via_mp_workspace_size bytes (too small:
    # MPGEMM_ENOMEM before any launch), and the same call on an SM partition
    import torch
    m, l, n, bits, depth = 72, 88, 56, 128, 2
    A = I.dd_random(m, l, 730, exp_spread=20)
    B = I.dd_random(l, n, 731, exp_spread=20)
    Co = oracle.gemm_via_mp(A, B, bits, algo="strassen", n_min=16, depth=depth)
    L = mpg.lib()
    need = L.mpgemm_via_mp_workspace_size(bits, m, l, n, 2, depth)
    assert need >= 4 * (2 + bits // 32) * (m * l + l * n + m * n)
    assert L.mpgemm_via_mp_workspace_size(96, m, l, n, 2, depth) == 0
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    try:
        mpg.set_workspace(ws)
        C = mpg.gemm_via_mp(dev(A), dev(B), bits, algo="strassen", n_min=16, depth=depth).cpu().numpy()
        assert np.array_equal(C.view(np.uint64), Co.view(np.uint64))
        mpg.set_workspace(ws[: need - 256])
        with pytest.raises(mpg.MpgemmError) as e:
            mpg.gemm_via_mp(dev(A), dev(B), bits, algo="strassen", n_min=16, depth=depth)
        assert e.value.status == -6
    finally:
        mpg.set_workspace(None)
    with mpg.Partition(24) as part:
        Ad, Bd = dev(A), dev(B)
        torch.cuda.synchronize()
        C = mpg.gemm_via_mp(Ad, Bd, bits, algo="strassen", n_min=16, depth=depth, stream=part.stream)
        assert mpg.stream_status(part.stream) == 0
        assert np.array_equal(C.cpu().numpy().view(np.uint64), Co.view(np.uint64))
