"""Python binding of libmpgemm: multiple-precision dense GEMM C := AB on a
GB300 (Kouya, arXiv:1710.01839, Section 2, Eqs 1-3).

Argument marshalling only: every step runs in the CUDA library's kernels.
If the compiled library is missing this module raises; there is no CPU
fallback.  PyTorch supplies device memory and the current stream.

Layouts (see include/mpgemm.h): DD tensors are float64 of shape (2, rows,
cols) [hi, lo]; QD float64 (4, rows, cols); multi-limb uint32-compatible
int32/uint32 tensors of shape (2 + w, rows, cols) with p = 32 w bits.
"""

from __future__ import annotations

import ctypes

from ._lib import (ALGO, KIND, MpgemmError, check, check_planes, int_dtypes, lib, lib_path,  # noqa: F401
                   require_cuda)

__all__ = ["gemm_dd", "gemm_qd", "gemm_mp", "gemm_split", "gemm_via_mp", "to_mp", "from_mp", "workspace_size", "set_workspace", "stream_status", "strerror",
           "Partition", "PrecisionChoice", "precision_log2_bound", "select_precision", "exponent_spread",
           "MpgemmError", "ALGO", "KIND", "lib", "lib_path"]


def _torch():
    import torch
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


_check_tensor = check_planes


def _operands(A, B, planes, dtypes):
    """Check the structure of A (planes, m, l) and B (planes, l, n); return
    (m, l, n)."""
    _check_tensor(A, planes, dtypes, "A")
    m, l = A.shape[1], A.shape[2]
    _check_tensor(B, planes, dtypes, "B", rows=l)
    return m, l, B.shape[2]


def _algo(a):
    return ALGO[a] if isinstance(a, str) else int(a)


def _ddqd(fn, planes, A, B, C, algo, n_min, depth, stream):
    torch = _torch()
    m, l, n = _operands(A, B, planes, (torch.float64,))
    if C is None:
        C = torch.empty((planes, m, n), dtype=torch.float64, device=A.device)
    _check_tensor(C, planes, (torch.float64,), "C", rows=m, cols=n)
    require_cuda(A=A, B=B, C=C)
    rc = fn(m, l, n, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(C.data_ptr()),
            _algo(algo), int(n_min), int(depth), _stream_ptr(stream))
    check(rc)
    return C


def gemm_dd(A, B, C=None, algo="block", n_min=0, depth=0, stream=None):
    """C := AB in double-double (mpgemm_dd)."""
    return _ddqd(lib().mpgemm_dd, 2, A, B, C, algo, n_min, depth, stream)


def gemm_qd(A, B, C=None, algo="block", n_min=0, depth=0, stream=None):
    """C := AB in quad-double (mpgemm_qd)."""
    return _ddqd(lib().mpgemm_qd, 4, A, B, C, algo, n_min, depth, stream)


def gemm_mp(A, B, prec_bits, C=None, algo="block", n_min=0, depth=0, stream=None):
    """C := AB in p-bit multi-limb floating point, p = prec_bits (mpgemm_mp)."""
    torch = _torch()
    w = prec_bits // 32
    m, l, n = _operands(A, B, 2 + w, int_dtypes())
    if C is None:
        C = torch.empty((2 + w, m, n), dtype=A.dtype, device=A.device)
    _check_tensor(C, 2 + w, int_dtypes(), "C", rows=m, cols=n)
    require_cuda(A=A, B=B, C=C)
    rc = lib().mpgemm_mp(m, l, n, int(prec_bits), ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                         ctypes.c_void_p(C.data_ptr()), _algo(algo), int(n_min), int(depth), _stream_ptr(stream))
    check(rc)
    return C


def gemm_via_mp(A, B, prec_bits=0, C=None, algo="block", n_min=0, depth=0, stream=None):
    """C := AB for DD (2 planes) or QD (4 planes) computed on the integer
    pipe in prec_bits-bit multi-limb arithmetic (mpgemm_dd_via_mp /
    mpgemm_qd_via_mp); prec_bits = 0 picks 128 for DD and 256 for QD."""
    torch = _torch()
    T = A.shape[0] if isinstance(A, torch.Tensor) and A.dim() == 3 else 0
    if T not in (2, 4):
        raise ValueError("A must hold 2 (DD) or 4 (QD) planes")
    _operands(A, B, T, (torch.float64,))
    bits = int(prec_bits) or (128 if T == 2 else 256)
    L = lib()
    fn = L.mpgemm_dd_via_mp if T == 2 else L.mpgemm_qd_via_mp
    return _ddqd(lambda *a: fn(*a[:6], bits, *a[6:]), T, A, B, C, algo, n_min, depth, stream)


def to_mp(X, prec_bits, Y=None, stream=None):
    """DD / QD planes X (T, rows, cols) -> multi-limb planes (2 + w, rows,
    cols), c = RN_p(...RN_p(x_0 + x_1)... + x_(T-1)) (mpgemm_terms_to_mp)."""
    torch = _torch()
    T = X.shape[0] if isinstance(X, torch.Tensor) and X.dim() == 3 else 0
    if T not in (2, 4):
        raise ValueError("X must hold 2 (DD) or 4 (QD) planes")
    _check_tensor(X, T, (torch.float64,), "X")
    w = int(prec_bits) // 32
    if Y is None:
        Y = torch.empty((2 + w, X.shape[1], X.shape[2]), dtype=torch.int32, device=X.device)
    _check_tensor(Y, 2 + w, int_dtypes(), "Y", rows=X.shape[1], cols=X.shape[2])
    require_cuda(X=X, Y=Y)
    check(lib().mpgemm_terms_to_mp(T, X.shape[1] * X.shape[2], ctypes.c_void_p(X.data_ptr()), int(prec_bits),
                                   ctypes.c_void_p(Y.data_ptr()), _stream_ptr(stream)))
    return Y


def from_mp(Y, prec_bits, terms, X=None, stream=None):
    """Multi-limb planes -> greedy expansion in `terms` doubles (2: DD,
    4: QD), x_t = RN_53(r), r -= x_t (mpgemm_mp_to_terms)."""
    torch = _torch()
    w = int(prec_bits) // 32
    if terms not in (2, 4):
        raise ValueError("terms must be 2 (DD) or 4 (QD)")
    _check_tensor(Y, 2 + w, int_dtypes(), "Y")
    if X is None:
        X = torch.empty((terms, Y.shape[1], Y.shape[2]), dtype=torch.float64, device=Y.device)
    _check_tensor(X, terms, (torch.float64,), "X", rows=Y.shape[1], cols=Y.shape[2])
    require_cuda(Y=Y, X=X)
    check(lib().mpgemm_mp_to_terms(int(terms), Y.shape[1] * Y.shape[2], int(prec_bits), ctypes.c_void_p(Y.data_ptr()),
                                   ctypes.c_void_p(X.data_ptr()), _stream_ptr(stream)))
    return X


def gemm_split(A, B, C=None, slices=0, digits="e4m3", stream=None):
    """Split-precision GEMM on the tensor cores: DD (2 planes; int8 or e4m3
    digits) or QD (4 planes; e4m3 digits).  slices = 0 picks the default
    (DD: 16 int8 / 22 e4m3; QD: 44)."""
    torch = _torch()
    T = A.shape[0] if isinstance(A, torch.Tensor) and A.dim() == 3 else 0
    if T not in (2, 4):
        raise ValueError("A must hold 2 (DD) or 4 (QD) planes")
    m, l, n = _operands(A, B, T, (torch.float64,))
    if C is None:
        C = torch.empty((T, m, n), dtype=torch.float64, device=A.device)
    else:
        _check_tensor(C, T, (torch.float64,), "C", rows=m, cols=n)
    require_cuda(A=A, B=B, C=C)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    if T == 4:
        if digits != "e4m3":
            raise ValueError("QD split precision uses e4m3 digits")
        check(lib().mpgemm_qd_ozaki(m, l, n, p(A), p(B), p(C), int(slices), _stream_ptr(stream)))
    else:
        kind = {"int8": 0, "e4m3": 1}[digits]
        check(lib().mpgemm_dd_ozaki_ex(m, l, n, p(A), p(B), p(C), int(slices), kind, _stream_ptr(stream)))
    return C


def workspace_size(kind, m, l, n, algo="strassen", depth=1, prec_bits=0):
    k = KIND[kind] if isinstance(kind, str) else int(kind)
    return int(lib().mpgemm_workspace_size(k, int(prec_bits), m, l, n, _algo(algo), int(depth)))


def set_workspace(tensor=None):
    """Hand the library a device buffer (a CUDA tensor) to use as workspace;
    None reverts to per-call stream-ordered allocation.  Keep the tensor
    alive while calls that may use it run."""
    if tensor is None:
        check(lib().mpgemm_set_workspace(None, 0))
    else:
        check(lib().mpgemm_set_workspace(ctypes.c_void_p(tensor.data_ptr()), tensor.numel() * tensor.element_size()))


MP_LEAVES = {"default": 0, "thread": 1, "team": 2}


def set_mp_leaf(leaf):
    """Select the kernel of multi-limb block GEMMs at 512-2048 bits:
    "thread" (one thread per output), "team" (W / 8 lanes per output, limbs
    across lanes) or "default"; returns the previous setting's name
    (mpgemm_set_mp_leaf)."""
    if leaf not in MP_LEAVES:
        raise ValueError(f"leaf must be one of {sorted(MP_LEAVES)}")
    prev = lib().mpgemm_set_mp_leaf(MP_LEAVES[leaf])
    check(min(prev, 0))
    return {v: k for k, v in MP_LEAVES.items()}[prev]


def stream_status(stream=None):
    return int(lib().mpgemm_stream_status(_stream_ptr(stream)))


def strerror(status):
    return lib().mpgemm_strerror(int(status)).decode()


SEL_METHOD = {0: "dd", 1: "qd", 2: "mp", 3: "ozaki_int8", 4: "ozaki_e4m3", 5: "ozaki_qd", 6: "dd_via_mp",
              7: "qd_via_mp"}
_SEL_CODE = {v: k for k, v in SEL_METHOD.items()}


class PrecisionChoice(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("prec_bits", ctypes.c_int), ("num_slices", ctypes.c_int),
                ("log2_bound", ctypes.c_double), ("est_ms", ctypes.c_double)]


def precision_log2_bound(method, l, prec_bits=0, num_slices=0, spread=0):
    """log2 of the a-priori elementwise bound |C - AB| <= beta |A||B| of one
    configuration (mpgemm_precision_log2_bound)."""
    return float(lib().mpgemm_precision_log2_bound(_SEL_CODE[method], int(prec_bits), int(num_slices), int(l),
                                                   int(spread)))


def select_precision(log2_target, m, l, n, spread=0, max_out=8):
    """Configurations whose bound meets 2^log2_target, fastest first
    (mpgemm_select_precision): a list of dicts."""
    out = (PrecisionChoice * max_out)()
    k = lib().mpgemm_select_precision(float(log2_target), int(m), int(l), int(n), int(spread), out, int(max_out))
    if k < 0:
        check(k)
    return [{"method": SEL_METHOD[c.method], "prec_bits": c.prec_bits, "num_slices": c.num_slices,
             "log2_bound": c.log2_bound, "est_ms": c.est_ms} for c in out[:min(k, max_out)]]


def exponent_spread(A, B, stream=None):
    """Binade spread of DD operands (mpgemm_dd_exponent_spread), computed on the GPU."""
    torch = _torch()
    _operands(A, B, 2, (torch.float64,))
    require_cuda(A=A, B=B)
    v = ctypes.c_int()
    check(lib().mpgemm_dd_exponent_spread(A.shape[1], A.shape[2], B.shape[2], ctypes.c_void_p(A.data_ptr()),
                                          ctypes.c_void_p(B.data_ptr()), ctypes.byref(v), _stream_ptr(stream)))
    return v.value


class Partition:
    """A stream whose kernels run on (at least) `num_sms` SMs: a CUDA green
    context made by mpgemm_partition_create.  `stream` is a
    torch.cuda.ExternalStream to pass as the `stream` argument of this
    module's calls; `sms` is the partition's actual SM count.  Synchronise
    with stream_status(p.stream); close() (or leaving a `with` block)
    synchronises and destroys it."""

    def __init__(self, num_sms):
        torch = _torch()
        h, n = ctypes.c_void_p(), ctypes.c_int()
        check(lib().mpgemm_partition_create(int(num_sms), ctypes.byref(h), ctypes.byref(n)))
        self.handle = h.value
        self.sms = n.value
        self.stream = torch.cuda.ExternalStream(self.handle)

    def close(self):
        if self.handle is not None:
            h, self.handle = self.handle, None
            check(lib().mpgemm_partition_destroy(ctypes.c_void_p(h)))

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
