"""The oracle: a plain, slow CPU reference for the multiple-precision GEMM
(Kouya, arXiv:1710.01839, Section 2, Eqs 1-3) and for the split-precision DD
GEMM steps.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library shares no code with it and never calls it.

The arithmetic lives in ``mpgemm_oracle.c`` (plain C, compiled with
``-ffp-contract=off``); this module compiles it (``build()``) and wraps it
with ctypes.  Parity of every function is pinned by the ``-m "not gpu"``
tests against exact rational arithmetic, mpmath, closed forms and the
paper's tables; ``tests/test_oracle_mutants.py`` plants mistakes in copies
of the C source and requires those pins to catch every one.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpgemm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")

ALGO = {"simple": 0, "block": 1, "strassen": 2}

_lib = None


def compile_source(src: str, out: str) -> str:
    """Compile one C source of the oracle into the shared library `out`."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    return compile_source(_SRC, _LIB)


def lib():
    """The compiled oracle.  MPGEMM_ORACLE_LIB names another compiled copy of
    mpgemm_oracle.c to load instead (the planted-mistake tests use it)."""
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(os.environ.get("MPGEMM_ORACLE_LIB") or build())
        _declare(_lib)
    return _lib


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double


def _declare(L):
    L.or_set_threads.argtypes = [_I]
    L.or_get_threads.restype = _I
    for name in ("or_two_sum", "or_fast_two_sum", "or_two_prod"):
        getattr(L, name).argtypes = [_D, _D, _P]
    for name in ("or_dd_add", "or_dd_mul", "or_qd_add", "or_qd_mul"):
        getattr(L, name).argtypes = [_P, _P, _P]
    L.or_round_terms.argtypes = [_P, _I, _P, _I]
    L.or_mp_mul.argtypes = [_I, _P, _P, _P]
    L.or_mp_add.argtypes = [_I, _P, _P, _P]
    L.or_terms_to_mp.argtypes = [_I, _I64, _P, _I, _P]
    L.or_mp_to_terms.argtypes = [_I, _I64, _I, _P, _P]
    for name in ("or_dd_gemm", "or_qd_gemm"):
        f = getattr(L, name)
        f.argtypes = [_I, _I64, _I64, _I64, _P, _P, _P, _I64, _I, _I64, _I64]
        f.restype = _I
    L.or_mp_gemm.argtypes = [_I, _I, _I64, _I64, _I64, _P, _P, _P, _I64, _I, _I64, _I64]
    L.or_mp_gemm.restype = _I
    L.or_exact_check.argtypes = [_I, _I64, _I64, _I64, _P, _P, _P, _I64, _P, _P, _P, _P]
    L.or_exact_check.restype = _I
    L.or_exact_entries.argtypes = [_I, _I64, _I64, _I64, _P, _P, _I64, _P, _P, _P]
    L.or_exact_entries.restype = _I
    L.or_ozaki_row_expo.argtypes = [_I64, _I64, _P, _P]
    L.or_ozaki_col_expo.argtypes = [_I64, _I64, _P, _P]
    L.or_ozaki_slice.argtypes = [_I, _I64, _I64, _P, _P, _I, _P]
    L.or_ozaki_levels.argtypes = [_I64, _I64, _I64, _I, _P, _P, _P]
    L.or_ozaki_recombine.argtypes = [_I64, _I64, _I, _P, _P, _P, _P]
    L.or_ozaki_gemm.argtypes = [_I64, _I64, _I64, _P, _P, _P, _I]
    L.or_ozaki_gemm.restype = _I
    L.or_ozaki_slice_b32.argtypes = [_I, _I64, _I64, _P, _P, _I, _P]
    L.or_ozaki_recombine_bits.argtypes = [_I64, _I64, _I, _I, _I, _P, _P, _P, _P]
    L.or_ozaki_gemm_b32.argtypes = [_I64, _I64, _I64, _P, _P, _P, _I]
    L.or_ozaki_gemm_b32.restype = _I
    L.or_ozaki_slice_b32_terms.argtypes = [_I, _I, _I64, _I64, _P, _P, _I, _P]
    L.or_ozaki_recombine_terms.argtypes = [_I64, _I64, _I, _I, _I, _I, _P, _P, _P, _P]
    L.or_ozaki_gemm_b32_terms.argtypes = [_I, _I64, _I64, _I64, _P, _P, _P, _I]
    L.or_ozaki_gemm_b32_terms.restype = _I


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(t: int) -> None:
    lib().or_set_threads(int(t))


def threads() -> int:
    return int(lib().or_get_threads())


# --------------------------------------------------------------------------
# scalar operations (for the pins)
# --------------------------------------------------------------------------

def two_sum(a: float, b: float):
    out = np.zeros(2)
    lib().or_two_sum(a, b, _ptr(out))
    return float(out[0]), float(out[1])


def fast_two_sum(a: float, b: float):
    out = np.zeros(2)
    lib().or_fast_two_sum(a, b, _ptr(out))
    return float(out[0]), float(out[1])


def two_prod(a: float, b: float):
    out = np.zeros(2)
    lib().or_two_prod(a, b, _ptr(out))
    return float(out[0]), float(out[1])


def _binop(name, x, y, n):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = np.zeros(n)
    getattr(lib(), name)(_ptr(x), _ptr(y), _ptr(z))
    return z


def dd_add(x, y):
    return _binop("or_dd_add", x, y, 2)


def dd_mul(x, y):
    return _binop("or_dd_mul", x, y, 2)


def qd_add(x, y):
    return _binop("or_qd_add", x, y, 4)


def qd_mul(x, y):
    return _binop("or_qd_mul", x, y, 4)


def round_terms(values, terms: int):
    v = np.ascontiguousarray(values, dtype=np.float64)
    out = np.zeros(terms)
    lib().or_round_terms(_ptr(v), len(v), _ptr(out), terms)
    return out


def mp_mul(w: int, x, y):
    x = np.ascontiguousarray(x, dtype=np.uint32)
    y = np.ascontiguousarray(y, dtype=np.uint32)
    z = np.zeros(2 + w, dtype=np.uint32)
    lib().or_mp_mul(w, _ptr(x), _ptr(y), _ptr(z))
    return z


def mp_add(w: int, x, y):
    x = np.ascontiguousarray(x, dtype=np.uint32)
    y = np.ascontiguousarray(y, dtype=np.uint32)
    z = np.zeros(2 + w, dtype=np.uint32)
    lib().or_mp_add(w, _ptr(x), _ptr(y), _ptr(z))
    return z


# --------------------------------------------------------------------------
# GEMM (Eqs 1-3)
# --------------------------------------------------------------------------

def _gemm(fn, A, B, dtype, planes, algo, n_min, depth, rows, extra=()):
    A = np.ascontiguousarray(A, dtype=dtype)
    B = np.ascontiguousarray(B, dtype=dtype)
    m, l = A.shape[1], A.shape[2]
    n = B.shape[2]
    assert B.shape[1] == l and A.shape[0] == planes and B.shape[0] == planes
    C = np.zeros((planes, m, n), dtype=dtype)
    r0, r1 = (0, m) if rows is None else rows
    rc = fn(*extra, ALGO[algo], m, l, n, _ptr(A), _ptr(B), _ptr(C), int(n_min), int(depth), int(r0), int(r1))
    if rc != 0:
        raise ValueError(f"oracle GEMM rejected the arguments (status {rc})")
    return C


def dd_gemm(A, B, algo="simple", n_min=64, depth=0, rows=None):
    return _gemm(lib().or_dd_gemm, A, B, np.float64, 2, algo, n_min, depth, rows)


def qd_gemm(A, B, algo="simple", n_min=64, depth=0, rows=None):
    return _gemm(lib().or_qd_gemm, A, B, np.float64, 4, algo, n_min, depth, rows)


def mp_gemm(A, B, prec_bits, algo="simple", n_min=64, depth=0, rows=None):
    w = prec_bits // 32
    return _gemm(lib().or_mp_gemm, A, B, np.uint32, 2 + w, algo, n_min, depth, rows, extra=(int(prec_bits),))


def terms_to_mp(X, prec_bits):
    """DD / QD planes (T, rows, cols) -> multi-limb planes (2 + w, rows,
    cols): c = +0, c = RN_p(c + x_t) for t = 0..T-1."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    T, r, c = X.shape
    w = prec_bits // 32
    Y = np.zeros((2 + w, r, c), dtype=np.uint32)
    lib().or_terms_to_mp(T, r * c, _ptr(X), w, _ptr(Y))
    return Y


def mp_to_terms(Y, prec_bits, terms):
    """Multi-limb planes -> the greedy expansion in `terms` doubles:
    x_t = RN_53(r), r = r - x_t."""
    w = prec_bits // 32
    Y = np.ascontiguousarray(Y, dtype=np.uint32)
    assert Y.shape[0] == 2 + w
    X = np.zeros((terms, Y.shape[1], Y.shape[2]))
    lib().or_mp_to_terms(terms, Y.shape[1] * Y.shape[2], w, _ptr(Y), _ptr(X))
    return X


def gemm_via_mp(A, B, prec_bits, algo="simple", n_min=64, depth=0):
    """DD / QD C := AB computed in prec_bits-bit multi-limb arithmetic: the
    conversions above around the multi-limb GEMM."""
    T = A.shape[0]
    Cm = mp_gemm(terms_to_mp(A, prec_bits), terms_to_mp(B, prec_bits), prec_bits, algo=algo, n_min=n_min,
                 depth=depth)
    return mp_to_terms(Cm, prec_bits, T)


def exact_check(A, B, C, ii, jj):
    """For sampled (i, j): (|c_exact - c|, sum_k |a_ik||b_kj|), exact then
    rounded; A, B, C hold 2 (DD) or 4 (QD) planes."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    C = np.ascontiguousarray(C, dtype=np.float64)
    terms = A.shape[0]
    m, l, n = A.shape[1], A.shape[2], B.shape[2]
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    err = np.zeros(len(ii))
    absab = np.zeros(len(ii))
    rc = lib().or_exact_check(terms, m, l, n, _ptr(A), _ptr(B), _ptr(C), len(ii), _ptr(ii), _ptr(jj),
                              _ptr(err), _ptr(absab))
    assert rc == 0
    return err, absab


def exact_entries(A, B, ii, jj, terms):
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    m, l, n = A.shape[1], A.shape[2], B.shape[2]
    ii = np.ascontiguousarray(ii, dtype=np.int64)
    jj = np.ascontiguousarray(jj, dtype=np.int64)
    out = np.zeros((len(ii), terms))
    rc = lib().or_exact_entries(A.shape[0], m, l, n, _ptr(A), _ptr(B), len(ii), _ptr(ii), _ptr(jj), _ptr(out))
    assert rc == 0
    return out


# --------------------------------------------------------------------------
# split-precision DD GEMM steps
# --------------------------------------------------------------------------

def ozaki_row_expo(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    e = np.zeros(A.shape[1], dtype=np.int32)
    lib().or_ozaki_row_expo(A.shape[1], A.shape[2], _ptr(A[0]), _ptr(e))
    return e


def ozaki_col_expo(B):
    B = np.ascontiguousarray(B, dtype=np.float64)
    f = np.zeros(B.shape[2], dtype=np.int32)
    lib().or_ozaki_col_expo(B.shape[1], B.shape[2], _ptr(np.ascontiguousarray(B[0])), _ptr(f))
    return f


def ozaki_slice(X, expo, S, by_col):
    X = np.ascontiguousarray(X, dtype=np.float64)
    expo = np.ascontiguousarray(expo, dtype=np.int32)
    D = np.zeros((S, X.shape[1], X.shape[2]), dtype=np.int8)
    lib().or_ozaki_slice(1 if by_col else 0, X.shape[1], X.shape[2], _ptr(X), _ptr(expo), S, _ptr(D))
    return D


def ozaki_levels(DA, DB, S):
    m, l = DA.shape[1], DA.shape[2]
    n = DB.shape[2]
    L = np.zeros((2 * S + 1, m, n), dtype=np.int64)
    lib().or_ozaki_levels(m, l, n, S, _ptr(np.ascontiguousarray(DA)), _ptr(np.ascontiguousarray(DB)), _ptr(L))
    return L


def ozaki_recombine(L, e, f, S):
    m, n = L.shape[1], L.shape[2]
    C = np.zeros((2, m, n))
    lib().or_ozaki_recombine(m, n, S, _ptr(np.ascontiguousarray(L)), _ptr(np.ascontiguousarray(e, dtype=np.int32)),
                             _ptr(np.ascontiguousarray(f, dtype=np.int32)), _ptr(C))
    return C


def ozaki_gemm(A, B, S):
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    m, l, n = A.shape[1], A.shape[2], B.shape[2]
    C = np.zeros((2, m, n))
    lib().or_ozaki_gemm(m, l, n, _ptr(A), _ptr(B), _ptr(C), S)
    return C


def ozaki_slice_b32(X, expo, S, by_col):
    """Balanced base-32 digits (|d| <= 16, FP8 e4m3-exact), S planes."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    expo = np.ascontiguousarray(expo, dtype=np.int32)
    D = np.zeros((S, X.shape[1], X.shape[2]), dtype=np.int8)
    lib().or_ozaki_slice_b32(1 if by_col else 0, X.shape[1], X.shape[2], _ptr(X), _ptr(expo), S, _ptr(D))
    return D


def ozaki_recombine_bits(L, e, f, S, bits, head):
    m, n = L.shape[1], L.shape[2]
    C = np.zeros((2, m, n))
    lib().or_ozaki_recombine_bits(m, n, S, bits, head, _ptr(np.ascontiguousarray(L)),
                                  _ptr(np.ascontiguousarray(e, dtype=np.int32)),
                                  _ptr(np.ascontiguousarray(f, dtype=np.int32)), _ptr(C))
    return C


def ozaki_gemm_b32(A, B, S):
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    m, l, n = A.shape[1], A.shape[2], B.shape[2]
    C = np.zeros((2, m, n))
    lib().or_ozaki_gemm_b32(m, l, n, _ptr(A), _ptr(B), _ptr(C), S)
    return C


def ozaki_slice_b32_terms(X, expo, S, by_col):
    """Balanced base-32 digits of a T-plane expansion (T = X.shape[0]: 2 DD,
    4 QD) from its exact sum: S planes (B not transposed)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    expo = np.ascontiguousarray(expo, dtype=np.int32)
    D = np.zeros((S, X.shape[1], X.shape[2]), dtype=np.int8)
    lib().or_ozaki_slice_b32_terms(1 if by_col else 0, X.shape[0], X.shape[1], X.shape[2], _ptr(X), _ptr(expo), S,
                                   _ptr(D))
    return D


def ozaki_recombine_terms(L, e, f, S, T, bits=5, head=1):
    m, n = L.shape[1], L.shape[2]
    C = np.zeros((T, m, n))
    lib().or_ozaki_recombine_terms(m, n, S, bits, head, T, _ptr(np.ascontiguousarray(L)),
                                   _ptr(np.ascontiguousarray(e, dtype=np.int32)),
                                   _ptr(np.ascontiguousarray(f, dtype=np.int32)), _ptr(C))
    return C


def ozaki_gemm_b32_terms(A, B, S):
    """The FP8-digit split-precision GEMM of T-term expansions (T = A.shape[0])."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    T, m, l, n = A.shape[0], A.shape[1], A.shape[2], B.shape[2]
    C = np.zeros((T, m, n))
    lib().or_ozaki_gemm_b32_terms(T, m, l, n, _ptr(A), _ptr(B), _ptr(C), S)
    return C
