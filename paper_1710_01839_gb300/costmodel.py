"""FP32 MLP cost model through the C ABI (mpgemm_cost_*): collect timings,
train, predict, save and load.  The kernels (training, inference) and the
timing sweep are in the library; this module only marshals arrays."""

from __future__ import annotations

import ctypes
import os

import numpy as np

from ._lib import KIND, check, lib

ALGO = {"simple": 0, "block": 1, "strassen": 2}
DEFAULT_MODEL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "cost_model_gb300.bin")


def num_features() -> int:
    return int(lib().mpgemm_cost_num_features())


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def features(kind, m, l, n, algo, tile, depth=0, prec_bits=0):
    k = KIND[kind] if isinstance(kind, str) else int(kind)
    a = ALGO[algo] if isinstance(algo, str) else int(algo)
    out = np.zeros(num_features(), dtype=np.float32)
    check(lib().mpgemm_cost_features(k, int(prec_bits), int(m), int(l), int(n), a, int(tile), int(depth), _ptr(out)))
    return out


def collect(count, seed=1714, max_dim=1024, stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    F = np.zeros((count, num_features()), dtype=np.float32)
    T = np.zeros(count, dtype=np.float32)
    check(lib().mpgemm_cost_collect(int(count), ctypes.c_ulonglong(seed), int(max_dim), _ptr(F), _ptr(T),
                                    ctypes.c_void_p(int(s.cuda_stream))))
    return F, T


def _rows_of_features(F, count=None):
    F = _f32(np.atleast_2d(F))
    if F.ndim != 2 or F.shape[1] != num_features() or (count is not None and F.shape[0] != count):
        want = f"({'count' if count is None else count}, {num_features()})"
        raise ValueError(f"feature rows must have shape {want}, got {F.shape}")
    return F


def train(F, T, epochs=200, seed=1714):
    T = _f32(T).reshape(-1)
    F = _rows_of_features(F, len(T))
    if int(epochs) <= 0:
        raise ValueError("epochs must be positive")
    loss = np.zeros(epochs, dtype=np.float32)
    check(lib().mpgemm_cost_train(_ptr(F), _ptr(T), len(T), int(epochs), ctypes.c_ulonglong(seed), _ptr(loss)))
    return loss


def predict(F):
    F = _rows_of_features(F)
    out = np.zeros(len(F), dtype=np.float32)
    check(lib().mpgemm_cost_predict(_ptr(F), len(F), _ptr(out)))
    return out


def save(path=DEFAULT_MODEL):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    check(lib().mpgemm_cost_save(path.encode()))


def load(path=DEFAULT_MODEL):
    check(lib().mpgemm_cost_load(path.encode()))


def clear():
    lib().mpgemm_cost_clear()


def choice(fmt, m, l, n, prec_bits=0, stream=None):
    """The installed model's (algo, n_min, depth) and predicted ms for a
    problem (mpgemm_cost_choice); None when no model is installed."""
    algo, nm, d, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
    sp = None if stream is None else ctypes.c_void_p(int(stream.cuda_stream))
    rc = lib().mpgemm_cost_choice(KIND["mp" if fmt.startswith("mp") else fmt], int(prec_bits), int(m), int(l), int(n),
                                  sp, ctypes.byref(algo), ctypes.byref(nm), ctypes.byref(d), ctypes.byref(ms))
    if rc == -2:
        return None
    check(rc)
    return {"algo": {0: "simple", 1: "block", 2: "strassen"}[algo.value], "n_min": nm.value, "depth": d.value,
            "pred_ms": ms.value}
