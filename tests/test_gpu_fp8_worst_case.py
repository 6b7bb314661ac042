"""Worst cases of the FP8 (e4m3) split-precision path: the tcgen05 tensor
cores accumulate the integer products of balanced base-32 digits (|d| <= 16)
in f32, and the level sums are exact only if every partial sum of a chunk
of Q = floor(2^24 / (256 lp)) slice pairs stays an exactly represented
integer.  Random digits keep the sums near sqrt(l) 10^2, far from 2^24, so
these tests drive the sums to the chunk bound itself, with digit planes
built directly (all +16 against +16, -16 against +16, 15 against 15 so that
every bit of a 24-bit sum is set, large products followed by products of 1
so that small addends meet an accumulator near 2^24), and compare the level
sums bit for bit with the oracle's integer level sums:

  * l = 65536: Q = 1, one slice pair's sum reaches 256 l = 2^24;
  * l = 4096 and l = 4000 (lp = 4096): Q = 16, Q 256 lp = 2^24 exactly, a
    chunk of 16 pairs reaches 2^24;
  * l = 65535 (lp = 65536): one pair's sum reaches 2^24 - 256;
  * l = 4992: Q = 13, a chunk just under 2^24 (Q 256 lp = 2^24 - 163840).

End to end, DD and QD inputs whose digits are (almost) all of magnitude 16
(the value sum_s d_s 32^-s with d_1 = 16, d_s = -16, at the top of its
row's / column's binade) go through mpgemm_dd_ozaki_ex / mpgemm_qd_ozaki and
must be bit-identical to the oracle."""

import ctypes
from fractions import Fraction

import numpy as np
import pytest

import oracle
from gpu_util import dev, host

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


def _e4m3_table():
    """code -> exact value for the 256 e4m3 codes (test helper; NaN codes
    excluded), and the canonical code of every integer in [-16, 16]."""
    c = np.arange(256, dtype=np.int64)
    sign = np.where(c & 0x80, -1.0, 1.0)
    e = (c >> 3) & 0xF
    mant = c & 7
    val = sign * np.where(e == 0, mant / 8.0 * 2.0**-6, (1 + mant / 8.0) * 2.0 ** (e - 7))
    enc = {}
    for v in range(-16, 17):
        codes = [int(k) for k in range(256) if (k & 0x7F) != 0x7F and val[k] == v]
        enc[v] = 0 if v == 0 else codes[0]
    return enc


ENC = _e4m3_table()


def _encode(D):
    out = np.zeros(D.shape, dtype=np.uint8)
    for v, code in ENC.items():
        out[D == v] = code
    return out


def _row_patterns(l, rng):
    """Rows of digits (values in [-16, 16]) that stress the accumulator."""
    k = np.arange(l)
    rows = [
        np.full(l, 16),                                  # all +16
        np.full(l, -16),                                 # all -16
        np.full(l, 15),                                  # 15: odd products, every bit of the sum set
        np.where(k < l - 64, 16, 1),                     # large products, then products of 1 / 15 / 16
        np.where(k % 33 == 32, 1, 16),                   # small products sprinkled into a large sum
        np.where(k == l - 1, 15, 16),                    # 256 (l - 1) + 225: odd, just under 256 l
        np.where(k < l // 2, 16, -16),                   # up to 2^23, then back to zero
        np.where(k < 64, 1, 16),                         # small first, then large
        rng.integers(-16, 17, size=l),                   # random
    ]
    return np.stack(rows).astype(np.int64)


def _col_patterns(l, rng):
    k = np.arange(l)
    cols = [
        np.full(l, 16),
        np.full(l, 15),
        np.full(l, 1),
        np.where(rng.integers(0, 2, size=l) == 1, 16, -16),
        np.where(k == l - 1, 15, 16),
        np.where(k % 2 == 0, 16, 15),
    ]
    return np.stack(cols, axis=1).astype(np.int64)   # (l, n)


def _levels_case(l, S, seed):
    """Digit planes (S, m, l) / (S, l, n): every slice carries the pattern,
    with its sign flipped on a seeded subset of slices."""
    import torch
    rng = np.random.default_rng(seed)
    ra, cb = _row_patterns(l, rng), _col_patterns(l, rng)
    m, n = ra.shape[0], cb.shape[1]
    sa = np.where(rng.integers(0, 4, size=S) == 0, -1, 1)
    sb = np.where(rng.integers(0, 4, size=S) == 0, -1, 1)
    sa[:2] = 1
    sb[:2] = 1
    DA = np.stack([sa[s] * ra for s in range(S)])             # (S, m, l)
    DB = np.stack([sb[s] * cb for s in range(S)])             # (S, l, n)
    lp = _lp(l)
    ga = np.zeros((S, m, lp), dtype=np.uint8)
    gb = np.zeros((S, n, lp), dtype=np.uint8)
    ga[:, :, :l] = _encode(DA)
    gb[:, :, :l] = _encode(DB.transpose(0, 2, 1))
    Lv = torch.zeros((S, m, n), dtype=torch.int32, device="cuda")
    DAd = torch.from_numpy(ga).cuda()
    DBd = torch.from_numpy(gb).cuda()
    rc = mpg.lib().mpgemm_ozaki_levels_ex(E4M3, m, l, n, S, _p(DAd), _p(DBd), _p(Lv), _sp())
    assert rc == 0, mpg.strerror(rc)
    want = oracle.ozaki_levels(DA.astype(np.int8), DB.astype(np.int8), S)[2:S + 2]
    return host(Lv).astype(np.int64), want, ra, cb


# (l, S): Q = floor(2^16 / lp) pairs per exact f32 chunk
@pytest.mark.parametrize("l,S", [(65536, 3), (65535, 3), (4096, 24), (4000, 24), (4992, 24), (4096, 17)])
def test_fp8_levels_at_the_chunk_bound(l, S):
    got, want, ra, cb = _levels_case(l, S, seed=l + S)
    lp = _lp(l)
    Q = (1 << 24) // (256 * lp)
    # the construction reaches the bound: some pair (all +16 x +16) sums to 256 l,
    # and with Q > 1 a chunk of Q such pairs sums to Q 256 lp
    assert int(ra[0] @ cb[:, 0]) == 256 * l
    peak = int(np.max(np.abs(want)))
    if Q == 1:
        assert peak >= 256 * l
    else:
        assert S >= Q + 1 and 256 * l * min(Q, S) <= (1 << 24)
    bad = np.argwhere(got != want)
    assert bad.size == 0, (f"{len(bad)} level sums differ; first (level index, i, j) = {bad[:4].tolist()}, "
                           f"got {[int(got[tuple(b)]) for b in bad[:4]]}, want {[int(want[tuple(b)]) for b in bad[:4]]}")


def test_fp8_levels_all_sixteen_full_tile():
    """A full 128 x 256 tile of all-+16 and all--16 digits at l = 65536: every
    accumulator of the tile sums to +-2^24 (Q = 1)."""
    import torch
    l, S, m, n = 65536, 2, 128, 256
    lp = _lp(l)
    sign_a = np.where(np.arange(m) % 2 == 0, 16, -16)
    ga = np.broadcast_to(np.array([ENC[int(v)] for v in sign_a], dtype=np.uint8)[None, :, None], (S, m, lp)).copy()
    gb = np.full((S, n, lp), ENC[16], dtype=np.uint8)
    Lv = torch.zeros((S, m, n), dtype=torch.int32, device="cuda")
    DAd, DBd = torch.from_numpy(ga).cuda(), torch.from_numpy(gb).cuda()
    rc = mpg.lib().mpgemm_ozaki_levels_ex(E4M3, m, l, n, S, _p(DAd), _p(DBd), _p(Lv), _sp())
    assert rc == 0
    got = host(Lv).astype(np.int64)
    row = (sign_a * 16 * l).astype(np.int64)
    # level g = 2: one pair; g = 3: two pairs (each its own chunk)
    assert np.array_equal(got[0], np.broadcast_to(row[:, None], (m, n)))
    assert np.array_equal(got[1], np.broadcast_to(2 * row[:, None], (m, n)))


def _max_digit_value(S):
    """sum_s d_s 32^-s with d_1 = 16 and d_s = -16 for s >= 2: the value in
    [1/4, 1/2) whose balanced base-32 digits all have magnitude 16."""
    return Fraction(16, 32) - sum(Fraction(16, 32**s) for s in range(2, S + 1))


def _expansion(v: Fraction, terms: int):
    out = []
    for _ in range(terms):
        x = float(v)
        out.append(x)
        v -= Fraction(x)
    return out


def _max_digit_matrix(rows, cols, terms, S, seed, by_col):
    """Every entry +-v 2^k with v of _max_digit_value(S), k fixed per row (A)
    or per column (B), so that every entry is at the top of its row's or
    column's binade; signs: all + in the first row / column, seeded after."""
    rng = np.random.default_rng(seed)
    t = np.array(_expansion(_max_digit_value(S), terms))
    scale = rng.integers(-12, 13, size=cols if by_col else rows)
    sign = np.where(rng.integers(0, 2, size=(rows, cols)) == 1, 1.0, -1.0)
    if by_col:
        sign[:, 0] = 1.0
        sc = np.ldexp(1.0, scale)[None, :]
    else:
        sign[0, :] = 1.0
        sc = np.ldexp(1.0, scale)[:, None]
    X = np.stack([t[q] * sign * sc for q in range(terms)])
    return np.ascontiguousarray(X)


def _check_digits_maximal(X, S, by_col, terms):
    expo = oracle.ozaki_col_expo(X) if by_col else oracle.ozaki_row_expo(X)
    if terms == 2:
        D = oracle.ozaki_slice_b32(X, expo, S, by_col)
    else:
        D = oracle.ozaki_slice_b32_terms(X, expo, S, by_col)
    frac16 = float(np.mean(np.abs(D.astype(np.int64)) == 16))
    assert frac16 >= 0.85, frac16
    return frac16


@pytest.mark.parametrize("l", [65536, 4096])
def test_fp8_dd_gemm_maximal_digits_bit_exact(l):
    import torch
    S, m, n = 22, 3, 2
    A = _max_digit_matrix(m, l, 2, S, seed=901, by_col=False)
    B = _max_digit_matrix(l, n, 2, S, seed=902, by_col=True)
    _check_digits_maximal(A, S, False, 2)
    _check_digits_maximal(B, S, True, 2)
    Ad, Bd = dev(A), dev(B)
    Cd = torch.empty((2, m, n), dtype=torch.float64, device="cuda")
    rc = mpg.lib().mpgemm_dd_ozaki_ex(m, l, n, _p(Ad), _p(Bd), _p(Cd), S, E4M3, _sp())
    assert rc == 0, mpg.strerror(rc)
    assert np.array_equal(host(Cd), oracle.ozaki_gemm_b32(A, B, S))


@pytest.mark.parametrize("l", [65536, 4096])
def test_fp8_qd_gemm_maximal_digits_bit_exact(l):
    import torch
    S, m, n = 44, 2, 2
    A = _max_digit_matrix(m, l, 4, S, seed=911, by_col=False)
    B = _max_digit_matrix(l, n, 4, S, seed=912, by_col=True)
    _check_digits_maximal(A, S, False, 4)
    _check_digits_maximal(B, S, True, 4)
    Ad, Bd = dev(A), dev(B)
    Cd = torch.empty((4, m, n), dtype=torch.float64, device="cuda")
    rc = mpg.lib().mpgemm_qd_ozaki(m, l, n, _p(Ad), _p(Bd), _p(Cd), S, _sp())
    assert rc == 0, mpg.strerror(rc)
    assert np.array_equal(host(Cd), oracle.ozaki_gemm_b32_terms(A, B, S))
