"""Batched uneven mixed-precision GEMMs through the C ABI
(mpgemm_batched_plan / _run / _run_graph / _sequential)."""

from __future__ import annotations

import ctypes

from ._lib import KIND, check, check_planes, int_dtypes, lib, require_cuda


class Desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("prec_bits", ctypes.c_int), ("m", ctypes.c_int64),
                ("l", ctypes.c_int64), ("n", ctypes.c_int64), ("A", ctypes.c_void_p), ("B", ctypes.c_void_p),
                ("C", ctypes.c_void_p), ("tile", ctypes.c_int), ("engine", ctypes.c_int)]


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(int(s.cuda_stream))


def make_descs(problems, tiles=None, integer_pipe=False):
    """problems: list of (fmt, A, B, C) with device tensors; fmt in
    {'dd', 'qd', 'mp256'}.  tiles: optional list of tile edges.
    integer_pipe: run the DD and QD problems on the integer pipe (128 / 256-bit
    limbs; engine = 1)."""
    import torch
    arr = (Desc * len(problems))()
    for i, (fmt, A, B, C) in enumerate(problems):
        kind = KIND["mp" if fmt.startswith("mp") else fmt]
        planes, dts = {0: (2, (torch.float64,)), 1: (4, (torch.float64,)), 2: (10, int_dtypes())}[kind]
        check_planes(A, planes, dts, f"A[{i}]")
        check_planes(B, planes, dts, f"B[{i}]", rows=A.shape[2])
        check_planes(C, planes, dts, f"C[{i}]", rows=A.shape[1], cols=B.shape[2])
        require_cuda(**{f"A[{i}]": A, f"B[{i}]": B, f"C[{i}]": C})
        engine = 1 if integer_pipe and kind != 2 else 0
        arr[i] = Desc(kind, 256 if kind == 2 else 0, A.shape[1], A.shape[2], B.shape[2], A.data_ptr(), B.data_ptr(),
                      C.data_ptr(), 0 if tiles is None else int(tiles[i]), engine)
    return arr


class Plan:
    def __init__(self, descs):
        self.descs = descs
        self.h = ctypes.c_void_p()
        check(lib().mpgemm_batched_plan(descs, len(descs), ctypes.byref(self.h)))

    def run(self, stream=None):
        check(lib().mpgemm_batched_run(self.h, _stream(stream)))

    def run_graph(self, stream=None):
        check(lib().mpgemm_batched_run_graph(self.h, _stream(stream)))

    def info(self):
        w, g = ctypes.c_int(), ctypes.c_int()
        t = (ctypes.c_int * len(self.descs))()
        check(lib().mpgemm_batched_info(self.h, ctypes.byref(w), ctypes.byref(g), t, len(self.descs)))
        return {"work_items": w.value, "grid": g.value, "tiles": list(t)}

    def close(self):
        if self.h:
            lib().mpgemm_batched_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sequential(descs, stream=None):
    check(lib().mpgemm_batched_sequential(descs, len(descs), _stream(stream)))
