"""The warp-cooperative multi-limb kernel (a team of w / 8 lanes per output,
8 limbs per lane; mpgemm_set_mp_leaf(MPGEMM_MP_LEAF_TEAM)) at 512, 1024 and
2048 bits: bit-identical to the oracle and to the one-thread-per-output
kernel on ragged shapes spanning several CTA tiles and K panels, on
structured limbs with ties and near-ties, on roundings that carry out of the
top limb, on sums that cancel (exactly, and in their leading bits with a
borrow), with zero operands mixed into every warp, as Strassen's leaves,
sampled at 128^3-256^3, and with the exponent-range flag."""

import numpy as np
import pytest

import oracle
from gpu_util import dev, host
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")

WIDTHS = [16, 32, 64]


@pytest.fixture(autouse=True)
def team_leaf():
    prev = mpg.set_mp_leaf("team")
    yield
    mpg.set_mp_leaf(prev)


def _both(A, B, p, **kw):
    """The team kernel's result and the one-thread kernel's on the same call."""
    Ad, Bd = dev(A), dev(B)
    Ct = host(mpg.gemm_mp(Ad, Bd, p, **kw), mp=True)
    prev = mpg.set_mp_leaf("thread")
    try:
        Cs = host(mpg.gemm_mp(Ad, Bd, p, **kw), mp=True)
    finally:
        mpg.set_mp_leaf(prev)
    return Ct, Cs


def _mp_planes(entries, w):
    """MP planes (2 + w, rows, cols) from a nested list of (sign, e, M)."""
    rows, cols = len(entries), len(entries[0])
    P = np.zeros((2 + w, rows, cols), dtype=np.uint32)
    for r in range(rows):
        for c in range(cols):
            sgn, e, M = entries[r][c]
            P[0, r, c] = np.int32(e).view(np.uint32)
            P[1, r, c] = sgn
            for q in range(w):
                P[2 + q, r, c] = (M >> (32 * q)) & 0xFFFFFFFF
    return P


@pytest.mark.parametrize("w", WIDTHS)
@pytest.mark.parametrize("m,l,n", [(37, 29, 23), (45, 70, 39), (1, 1, 1), (9, 17, 33)])
def test_team_ragged_bit_exact(w, m, l, n):
    A, B = I.mp_random(m, l, w, 500 + w + m), I.mp_random(l, n, w, 600 + w + n)
    Ct, Cs = _both(A, B, 32 * w, algo="block", n_min=16)
    assert np.array_equal(Ct, oracle.mp_gemm(A, B, prec_bits=32 * w))
    assert np.array_equal(Ct, Cs)
    assert mpg.stream_status() == 0


@pytest.mark.parametrize("w", WIDTHS)
def test_team_close_exponents_and_zeros(w):
    # exponents in [-2, 2] (many sums align within one limb in every team of
    # a warp, and many within several), every fifth entry zero, two rows of
    # B negatives of each other (exact cancellations)
    m, l, n = 21, 26, 19
    A = I.mp_random(m, l, w, 700 + w, emin=-2, emax=2)
    B = I.mp_random(l, n, w, 800 + w, emin=-2, emax=2)
    rng = np.random.default_rng(900 + w)
    zA = rng.random((m, l)) < 0.2
    A[:, zA] = 0
    A[1, zA] = 2 + rng.integers(0, 2, size=int(zA.sum()))     # +0 and -0
    B[:, 5, :] = B[:, 4, :]
    B[1, 5, :] ^= 1
    Ct, Cs = _both(A, B, 32 * w, algo="block", n_min=16)
    assert np.array_equal(Ct, oracle.mp_gemm(A, B, prec_bits=32 * w))
    assert np.array_equal(Ct, Cs)


@pytest.mark.parametrize("w", WIDTHS)
def test_team_equal_exponents(w):
    # every exponent 0: products and sums of operands of one binade
    m, l, n = 16, 24, 16
    A = I.mp_random(m, l, w, 1000 + w, emin=0, emax=0)
    B = I.mp_random(l, n, w, 1100 + w, emin=0, emax=0)
    Ct, _ = _both(A, B, 32 * w, algo="block", n_min=16)
    assert np.array_equal(Ct, oracle.mp_gemm(A, B, prec_bits=32 * w))


@pytest.mark.parametrize("w", WIDTHS)
def test_team_structured_ties(w):
    p = 32 * w
    m, l, n = 19, 21, 17
    rng = np.random.default_rng(4100 + w)
    A, B = I.mp_structured(m, l, w, 4200 + w), I.mp_structured(l, n, w, 4300 + w)
    tie_makers = [(1 << (p - 1)) + 1, 3 << (p - 2), (1 << (p - 1)) + 3, (1 << p) - 1, 1 << (p - 1),
                  (1 << (p - 1)) + (1 << (p // 2))]
    for P, shape in ((A, (m, l)), (B, (l, n))):
        mask = rng.random(shape) < 0.5
        for r, c in zip(*np.nonzero(mask)):
            v = tie_makers[int(rng.integers(0, len(tie_makers)))]
            for q in range(w):
                P[2 + q, r, c] = (v >> (32 * q)) & 0xFFFFFFFF
    Ct, Cs = _both(A, B, p, algo="block", n_min=16)
    assert np.array_equal(Ct, oracle.mp_gemm(A, B, prec_bits=p))
    assert np.array_equal(Ct, Cs)


@pytest.mark.parametrize("w", WIDTHS)
def test_team_round_carry_out(w):
    # a product just below 2^(2p-1) that rounds up to 2^(2p-1), and sums
    # 1 - 2^-p + (over half an ulp | an exact tie with odd M) rounding to 1
    p = 32 * w
    x = (1 << (p - 1)) + 12345
    while True:
        y = ((1 << (2 * p - 1)) - 1) // x
        if 0 < (1 << (2 * p - 1)) - x * y <= (1 << (p - 2)) and y >= (1 << (p - 1)):
            break
        x += 1
    one = (0, 1, 1 << (p - 1))
    ones = (0, 0, (1 << p) - 1)
    over_half = (0, -p, (1 << (p - 1)) + 1)
    tie = (0, -p, 1 << (p - 1))
    zero = (0, 0, 0)
    A = _mp_planes([[(0, 0, x), zero], [ones, over_half], [ones, tie]], w)
    A[1, 0, 1] = 2
    B = _mp_planes([[(0, 0, y), one], [one, one]], w)
    Ct, _ = _both(A, B, p, algo="block", n_min=16)
    assert np.array_equal(Ct, oracle.mp_gemm(A, B, prec_bits=p))
    top = Ct[2 + w - 1].astype(np.int64)
    low = Ct[2:2 + w - 1].astype(np.int64)
    for (r, c), e in (((0, 0), 0), ((1, 1), 1), ((2, 1), 1)):
        assert Ct[0, r, c].view(np.int32) == e and top[r, c] == 0x80000000 and not low[:, r, c].any()


@pytest.mark.parametrize("w", WIDTHS)
def test_team_cancellation_of_leading_bits(w):
    # c = x, then c + (-(x + delta)) with the same exponent: a borrow (the
    # difference is negated) and a cancellation of all but the low bits
    # (normalisation by up to p - 1 bits), for deltas at every limb
    p = 32 * w
    rng = np.random.default_rng(1200 + w)
    deltas = [1, 3, 1 << 31, 1 << 32, (1 << 40) + 7, 1 << (p // 2), (1 << (p - 3)) - 1, 1 << (p - 3)]
    one = (0, 1, 1 << (p - 1))
    rows = []
    for dlt in deltas:
        x = (1 << (p - 1)) + int(rng.integers(0, 1 << 30))
        rows.append([(0, 0, x), (1, 0, x + dlt), (0, -5, (1 << (p - 1)) + 1)])
    A = _mp_planes(rows, w)
    B = _mp_planes([[one, one], [one, one], [one, (0, 0, 0)]], w)
    B[1, 2, 1] = 2
    Ct, Cs = _both(A, B, p, algo="block", n_min=16)
    assert np.array_equal(Ct, oracle.mp_gemm(A, B, prec_bits=p))
    assert np.array_equal(Ct, Cs)


@pytest.mark.parametrize("w", WIDTHS)
@pytest.mark.parametrize("depth", [1, 2])
def test_team_strassen_leaves(w, depth):
    n = 40
    A, B = I.mp_random(n, n, w, 1300 + w), I.mp_random(n, n, w, 1400 + w)
    Ct, Cs = _both(A, B, 32 * w, algo="strassen", n_min=16, depth=depth)
    assert np.array_equal(Ct, oracle.mp_gemm(A, B, prec_bits=32 * w, algo="strassen", n_min=16, depth=depth))
    assert np.array_equal(Ct, Cs)


@pytest.mark.parametrize("w,n", [(16, 256), (32, 256), (64, 128)])
def test_team_large_sampled_rows(w, n):
    A = I.mp_random(n, n, w, I.seed_for(2, w))
    B = I.mp_random(n, n, w, I.seed_for(2, 100 + w))
    C = host(mpg.gemm_mp(dev(A), dev(B), 32 * w, algo="block", n_min=64), mp=True)
    for r0 in (0, n // 2 + 1, n - 1):
        Co = oracle.mp_gemm(A, B, prec_bits=32 * w, rows=(r0, r0 + 1))
        assert np.array_equal(C[:, r0], Co[:, r0]), r0


@pytest.mark.parametrize("w", WIDTHS)
def test_team_exponent_range_is_flagged(w):
    p = 32 * w
    top = 2 ** 31 - 1
    one = (0, 1, 1 << (p - 1))
    cases = {
        "mul_over": ([[(0, top - 5, 1 << (p - 1))]], [[(0, 10, 1 << (p - 1))]]),
        "mul_under": ([[(1, -2 ** 31 + 5, 1 << (p - 1))]], [[(0, -10, 1 << (p - 1))]]),
        "add_carry": ([[(0, top, (1 << p) - 1), (0, top - p, (1 << (p - 1)) + 1)]], [[one], [one]]),
        "in_range": ([[(0, top - 20, 1 << (p - 1))]], [[(0, 10, 1 << (p - 1))]]),
    }
    for name, (a, b) in cases.items():
        A, B = _mp_planes(a, w), _mp_planes(b, w)
        mpg.gemm_mp(dev(A), dev(B), p, algo="block", n_min=16)
        want = 0 if name == "in_range" else -4
        assert mpg.stream_status() == want, name


def test_default_leaf_follows_the_grid():
    import ctypes
    import torch
    mpg.set_mp_leaf("default")
    L = mpg.lib()
    sms = L.mpgemm_stream_sms(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert L.mpgemm_mp_leaf_choice(2048, 64, 64, 1, sms) == 2
    assert L.mpgemm_mp_leaf_choice(2048, 512, 512, 1, sms) == 1
    A, B = I.mp_random(40, 50, 64, 1500), I.mp_random(50, 30, 64, 1501)
    Cd = host(mpg.gemm_mp(dev(A), dev(B), 2048, algo="block", n_min=16), mp=True)
    Ct, Cs = _both(A, B, 2048, algo="block", n_min=16)
    assert np.array_equal(Cd, Ct) and np.array_equal(Cd, Cs)
    assert np.array_equal(Cd, oracle.mp_gemm(A, B, prec_bits=2048))
