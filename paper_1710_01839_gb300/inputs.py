"""Seeded synthetic inputs for the multiple-precision GEMM, shared by the
oracle tests, the CUDA parity tests and the benchmark.

This module holds input *generation* only: random draws, exact power-of-two
scaling, re-representation of a drawn value in canonical (non-overlapping)
form, and rounding of the paper's closed-form test matrices to a format.  It
contains none of the GEMM arithmetic.

Layouts (row-major planes, the library's ABI):
  DD  float64 array of shape (2, rows, cols): [hi, lo]
  QD  float64 array of shape (4, rows, cols): [x0, x1, x2, x3]
  MP  uint32  array of shape (2 + w, rows, cols):
      [exponent (int32 bits), flags (bit0 sign, bit1 zero), limb 0 .. limb w-1]
      value = (-1)^sign * M * 2^(exponent - 32 w), M = sum_i limb_i 2^(32 i),
      M in [2^(32w - 1), 2^(32w)).

Recipes (seed = 1710 + 100 * config + rep unless a test says otherwise):
  * DD (small-size config): hi ~ U[-1, 1], lo = hi * 2^-53 * u, u ~ U[-1, 1];
    the pair is then re-represented so that |lo| <= ulp(hi)/2 (same value).
  * DD/QD (large-size config): as above, both words scaled by 2^k per element,
    k ~ U{-20..20}.
  * QD limbs: x0 ~ U[-1, 1], x_{i+1} = x_i * 2^-53 * u_i, then re-represented
    non-overlapping.
  * MP: random sign, mantissa bits uniform with the top bit set, exponent
    ~ U{-64..64}.
  * Split-precision config: DD entries with A's rows scaled by 2^{r_i} and
    B's columns by 2^{c_j}, r, c ~ U{-16..16}.
  * The paper's matrices (Section 4): A = [sqrt(5)(i + j - 1)],
    B = [sqrt(3)(n - i)], i, j = 1..n, rounded to the format.
"""

from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

SEED_BASE = 1710


def seed_for(config: int, rep: int = 0) -> int:
    return SEED_BASE + 100 * config + rep


# ----------------------------------------------------------------------------
# canonical (non-overlapping) re-representation of a pair of doubles
# ----------------------------------------------------------------------------

def _canon_pair(hi: np.ndarray, lo: np.ndarray):
    """Rewrite (hi, lo) as (hi', lo') with hi' + lo' == hi + lo exactly and
    |lo'| <= ulp(hi')/2: hi' = RN(hi + lo) and lo' its exact rounding error
    (Knuth's TwoSum, six IEEE double operations, no precondition).  Only the
    representation changes, not the value; a pair that is already canonical
    is returned unchanged (outside exact half-ulp ties)."""
    s = hi + lo
    bv = s - hi
    av = s - bv
    return s, (hi - av) + (lo - bv)


def _canon_terms(x: np.ndarray) -> np.ndarray:
    """Apply the pairwise rule top-down until every adjacent pair is canonical
    (a rewrite of one pair can unsettle the pair above it, hence the passes;
    each pass moves value upward, and a few passes settle every element)."""
    x = x.copy()
    for _ in range(64):
        changed = False
        for i in range(x.shape[0] - 1):
            h, l = _canon_pair(x[i], x[i + 1])
            if not (np.array_equal(h, x[i]) and np.array_equal(l, x[i + 1])):
                changed = True
            x[i], x[i + 1] = h, l
        if not changed:
            return x
    raise RuntimeError("expansion did not settle")


# ----------------------------------------------------------------------------
# random matrices
# ----------------------------------------------------------------------------

def dd_random(rows: int, cols: int, seed: int, exp_spread: int = 0) -> np.ndarray:
    """DD planes (2, rows, cols): hi ~ U[-1,1], lo = hi 2^-53 u."""
    rng = np.random.default_rng(seed)
    hi = rng.uniform(-1.0, 1.0, size=(rows, cols))
    u = rng.uniform(-1.0, 1.0, size=(rows, cols))
    lo = np.ldexp(hi, -53) * u
    hi, lo = _canon_pair(hi, lo)
    out = np.stack([hi, lo])
    if exp_spread:
        k = rng.integers(-exp_spread, exp_spread + 1, size=(rows, cols))
        out = np.ldexp(out, k[None, :, :])
    return np.ascontiguousarray(out)


def qd_random(rows: int, cols: int, seed: int, exp_spread: int = 0) -> np.ndarray:
    """QD planes (4, rows, cols): x0 ~ U[-1,1], x_{i+1} = x_i 2^-53 u_i."""
    rng = np.random.default_rng(seed)
    x = np.empty((4, rows, cols))
    x[0] = rng.uniform(-1.0, 1.0, size=(rows, cols))
    for i in range(3):
        u = rng.uniform(-1.0, 1.0, size=(rows, cols))
        x[i + 1] = np.ldexp(x[i], -53) * u
    x = _canon_terms(x)
    if exp_spread:
        k = rng.integers(-exp_spread, exp_spread + 1, size=(rows, cols))
        x = np.ldexp(x, k[None, :, :])
    return np.ascontiguousarray(x)


def mp_random(rows: int, cols: int, w: int, seed: int, emin: int = -64, emax: int = 64) -> np.ndarray:
    """MP planes (2 + w, rows, cols) with uniform mantissa bits (top bit set)."""
    rng = np.random.default_rng(seed)
    out = np.empty((2 + w, rows, cols), dtype=np.uint32)
    out[0] = rng.integers(emin, emax + 1, size=(rows, cols)).astype(np.int32).view(np.uint32)
    out[1] = rng.integers(0, 2, size=(rows, cols), dtype=np.uint32)
    out[2:] = rng.integers(0, 2**32, size=(w, rows, cols), dtype=np.uint64).astype(np.uint32)
    out[2 + w - 1] |= np.uint32(0x80000000)
    return out


def mp_structured(rows: int, cols: int, w: int, seed: int, emin: int = -8, emax: int = 8) -> np.ndarray:
    """MP planes like mp_random, but every limb drawn from {0, 1, 2^31 - 1,
    2^31, 2^32 - 1, uniform}: products with long runs of zeros or ones,
    near-ties and exact ties below the rounding position."""
    rng = np.random.default_rng(seed)
    out = np.empty((2 + w, rows, cols), dtype=np.uint32)
    out[0] = rng.integers(emin, emax + 1, size=(rows, cols)).astype(np.int32).view(np.uint32)
    out[1] = rng.integers(0, 2, size=(rows, cols), dtype=np.uint32)
    special = np.array([0, 1, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF], dtype=np.uint64)
    pick = rng.integers(0, 6, size=(w, rows, cols))
    uni = rng.integers(0, 2**32, size=(w, rows, cols), dtype=np.uint64)
    out[2:] = np.where(pick < 5, special[np.minimum(pick, 4)], uni).astype(np.uint32)
    out[2 + w - 1] |= np.uint32(0x80000000)
    return out


def dd_rowcol_scaled(m: int, l: int, n: int, seed: int, spread: int = 16, inner_spread: int = 0):
    """Split-precision workload: DD A (m x l) with row i scaled by 2^{r_i},
    DD B (l x n) with column j scaled by 2^{c_j}; optional inner-dimension
    spread (A's columns and B's rows scaled by 2^{q_k})."""
    rng = np.random.default_rng(seed)
    A = dd_random(m, l, seed + 1)
    B = dd_random(l, n, seed + 2)
    r = rng.integers(-spread, spread + 1, size=m)
    c = rng.integers(-spread, spread + 1, size=n)
    A = np.ldexp(A, r[None, :, None])
    B = np.ldexp(B, c[None, None, :])
    if inner_spread:
        q = rng.integers(-inner_spread, inner_spread + 1, size=l)
        A = np.ldexp(A, q[None, None, :])
        B = np.ldexp(B, q[None, :, None])
    return np.ascontiguousarray(A), np.ascontiguousarray(B)


def qd_rowcol_scaled(m: int, l: int, n: int, seed: int, spread: int = 16):
    """Split-precision QD workload: QD A (m x l) with row i scaled by 2^{r_i},
    QD B (l x n) with column j scaled by 2^{c_j}, r, c ~ U{-spread..spread}."""
    rng = np.random.default_rng(seed)
    A = qd_random(m, l, seed + 1)
    B = qd_random(l, n, seed + 2)
    r = rng.integers(-spread, spread + 1, size=m)
    c = rng.integers(-spread, spread + 1, size=n)
    return (np.ascontiguousarray(np.ldexp(A, r[None, :, None])),
            np.ascontiguousarray(np.ldexp(B, c[None, None, :])))


# ----------------------------------------------------------------------------
# integer-valued matrices (exact in every format)
# ----------------------------------------------------------------------------

def int_matrix(rows: int, cols: int, seed: int, lo: int = -8, hi: int = 8) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(rows, cols)).astype(np.int64)


def ints_to_dd(v: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.stack([v.astype(np.float64), np.zeros(v.shape)]))


def ints_to_qd(v: np.ndarray) -> np.ndarray:
    z = np.zeros(v.shape)
    return np.ascontiguousarray(np.stack([v.astype(np.float64), z, z, z]))


def ints_to_mp(v: np.ndarray, w: int) -> np.ndarray:
    out = np.zeros((2 + w,) + v.shape, dtype=np.uint32)
    p = 32 * w
    flat = v.reshape(-1)
    planes = out.reshape(2 + w, -1)
    for idx, x in enumerate(flat.tolist()):
        if x == 0:
            planes[1, idx] = 2
            continue
        a = abs(int(x))
        L = a.bit_length()
        M = a << (p - L)
        planes[0, idx] = np.int32(L).view(np.uint32)
        planes[1, idx] = 1 if x < 0 else 0
        for i in range(w):
            planes[2 + i, idx] = (M >> (32 * i)) & 0xFFFFFFFF
    return out


# ----------------------------------------------------------------------------
# the paper's test matrices (Section 4)
# ----------------------------------------------------------------------------

_F = 1400  # bits of the fixed-point square roots used for rounding


def _sqrt_fixed(c: int, k: int) -> Fraction:
    """floor(k sqrt(c) 2^F) / 2^F, within 2^-F of k sqrt(c) (k >= 0)."""
    return Fraction(math.isqrt(c * k * k << (2 * _F)), 1 << _F)


def _terms_of(x: Fraction, nterms: int):
    out = []
    for _ in range(nterms):
        t = float(x)          # correctly rounded (CPython int/int division)
        out.append(t)
        x -= Fraction(t)
    return out


def _mp_of(c: int, k: int, w: int):
    """(exp, flags, limbs) of RN_p(k sqrt(c)); k sqrt(c) is irrational or an
    integer, never a rounding tie at these precisions."""
    p = 32 * w
    if k == 0:
        return 0, 2, [0] * w
    # e with 2^(e-1) <= k sqrt(c) < 2^e, i.e. 4^(e-1) <= c k^2 < 4^e
    v = c * k * k
    e = (v.bit_length() + 1) // 2
    while (1 << (2 * e)) <= v:
        e += 1
    while (1 << (2 * (e - 1))) > v:
        e -= 1
    shift = p - e + 2  # two extra bits
    if shift >= 0:
        X = math.isqrt(c * k * k << (2 * shift))
        exact = X * X == (c * k * k << (2 * shift))
    else:
        raise ValueError("value too large")
    M, extra = X >> 2, X & 3
    sticky = not exact
    if extra > 2 or (extra == 2 and (sticky or (M & 1))):
        M += 1
    if M >> p:
        M >>= 1
        e += 1
    limbs = [(M >> (32 * i)) & 0xFFFFFFFF for i in range(w)]
    return e, 0, limbs


def paper_matrices(n: int, fmt: str, w: int = 0):
    """A = [sqrt(5)(i+j-1)], B = [sqrt(3)(n-i)] rounded to fmt ('dd', 'qd',
    'mp' with w limbs), i, j = 1..n (Section 4)."""
    if fmt in ("dd", "qd"):
        T = 2 if fmt == "dd" else 4
        a_vals = {k: _terms_of(_sqrt_fixed(5, k), T) for k in range(1, 2 * n)}
        b_vals = {k: _terms_of(_sqrt_fixed(3, k), T) for k in range(0, n)}
        A = np.empty((T, n, n))
        B = np.empty((T, n, n))
        for i in range(1, n + 1):
            for j in range(1, n + 1):
                A[:, i - 1, j - 1] = a_vals[i + j - 1]
                B[:, i - 1, j - 1] = b_vals[n - i]
        return A, B
    if fmt == "mp":
        a_vals = {k: _mp_of(5, k, w) for k in range(1, 2 * n)}
        b_vals = {k: _mp_of(3, k, w) for k in range(0, n)}
        A = np.empty((2 + w, n, n), dtype=np.uint32)
        B = np.empty((2 + w, n, n), dtype=np.uint32)
        for i in range(1, n + 1):
            for j in range(1, n + 1):
                for M, vals, key in ((A, a_vals, i + j - 1), (B, b_vals, n - i)):
                    e, fl, limbs = vals[key]
                    M[0, i - 1, j - 1] = np.int32(e).view(np.uint32)
                    M[1, i - 1, j - 1] = fl
                    M[2:, i - 1, j - 1] = limbs
        return A, B
    raise ValueError(fmt)


def paper_closed_form(n: int, i: int) -> Fraction:
    """c_ij / sqrt(15) for the paper's matrices: sum_k (i+k-1)(n-k) =
    n(n-1)(3i+n-2)/6, the same for every j (i is 1-based)."""
    return Fraction(n * (n - 1) * (3 * i + n - 2), 6)


# ----------------------------------------------------------------------------
# the batched uneven workload
# ----------------------------------------------------------------------------

def batched_shapes(count: int = 512, seed: int = SEED_BASE + 4, lo: int = 16, hi: int = 1024):
    """(m, l, n, precision) per GEMM: log-uniform dims in [lo, hi], precision
    uniform over {'dd', 'qd', 'mp256'}."""
    rng = np.random.default_rng(seed)
    dims = np.exp(rng.uniform(math.log(lo), math.log(hi), size=(count, 3)))
    dims = np.clip(np.rint(dims).astype(np.int64), lo, hi)
    prec = rng.integers(0, 3, size=count)
    names = ["dd", "qd", "mp256"]
    return [(int(d[0]), int(d[1]), int(d[2]), names[int(p)]) for d, p in zip(dims, prec)]
