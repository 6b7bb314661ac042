"""The tuning step (Section 3) through the C ABI: mpgemm_tune."""

from __future__ import annotations

import ctypes
import math
import os

from ._lib import KIND, check, check_planes, int_dtypes, lib, require_cuda

ALGO_NAME = {0: "simple", 1: "block", 2: "strassen", 3: "auto"}
VERIFY, REMEMBER, SKIP_SIMPLE, QUICK, FORCE = 1, 2, 4, 8, 16


class TuneReport(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int), ("n_min", ctypes.c_int), ("depth", ctypes.c_int),
                ("best_ms", ctypes.c_double), ("n_cand", ctypes.c_int),
                ("cand_n_min", ctypes.c_int * 8), ("cand_rows", ctypes.c_int64 * 8),
                ("cand_sample_ms", ctypes.c_double * 8), ("cand_pred_ms", ctypes.c_double * 8),
                ("cand_full_ms", ctypes.c_double * 8), ("simple_ms", ctypes.c_double),
                ("block_ms", ctypes.c_double), ("strassen_ms", ctypes.c_double * 5),
                ("tuning_ms", ctypes.c_double), ("measured", ctypes.c_int), ("from_cache", ctypes.c_int)]


def _nan(x):
    return None if x is None or (isinstance(x, float) and math.isnan(x)) else x


def report_dict(r: TuneReport):
    cands = []
    for i in range(r.n_cand):
        full = _nan(r.cand_full_ms[i])
        pred = r.cand_pred_ms[i]
        cands.append({"n_min": r.cand_n_min[i], "rows": r.cand_rows[i], "sample_ms": r.cand_sample_ms[i],
                      "pred_ms": pred, "full_ms": full,
                      "rel_diff": (abs(pred - full) / full) if full else None})
    out = {"algo": ALGO_NAME[r.algo], "n_min": r.n_min, "depth": r.depth, "best_ms": r.best_ms,
           "candidates": cands, "simple_ms": _nan(r.simple_ms), "block_ms": r.block_ms,
           "strassen_ms": {d: _nan(r.strassen_ms[d]) for d in (1, 2, 3, 4)}, "tuning_ms": r.tuning_ms,
           "measured": r.measured, "from_cache": bool(r.from_cache)}
    # Section 3's claim: tuning costs 1.6-2.3x more without the prediction.
    # Device time of the procedure with the sampled runs vs. with full runs
    # of the block algorithm for every n_min (the final timings are common).
    if cands and all(c["full_ms"] is not None for c in cands):
        common = sum(v for v in [out["simple_ms"], out["block_ms"]] + list(out["strassen_ms"].values())
                     if v is not None)
        with_pred = sum(c["sample_ms"] for c in cands) + common
        without = sum(c["full_ms"] for c in cands) + common
        out["tuning_cost_ratio_without_prediction"] = without / with_pred
        out["max_prediction_rel_diff"] = max(c["rel_diff"] for c in cands)
    return out


def tune(fmt, A, B, C, flags=REMEMBER, prec_bits=0, stream=None):
    """Run mpgemm_tune on device tensors; returns (choice dict, report dict)."""
    import torch
    kind = KIND["mp" if fmt.startswith("mp") else fmt]
    if kind == KIND["mp"]:
        if int(prec_bits) <= 0 or int(prec_bits) % 32:
            raise ValueError("multi-limb tuning needs prec_bits, a positive multiple of 32")
        planes, dts = 2 + int(prec_bits) // 32, int_dtypes()
    else:
        planes, dts = (2 if kind == KIND["dd"] else 4), (torch.float64,)
    check_planes(A, planes, dts, "A")
    m, l = A.shape[1], A.shape[2]
    check_planes(B, planes, dts, "B", rows=l)
    n = B.shape[2]
    check_planes(C, planes, dts, "C", rows=m, cols=n)
    require_cuda(A=A, B=B, C=C)
    if stream is None:
        stream = torch.cuda.current_stream()
    rep = TuneReport()
    rc = lib().mpgemm_tune(kind, int(prec_bits), m, l, n, ctypes.c_void_p(A.data_ptr()),
                           ctypes.c_void_p(B.data_ptr()), ctypes.c_void_p(C.data_ptr()), int(flags),
                           ctypes.c_void_p(int(stream.cuda_stream)), ctypes.byref(rep))
    check(rc)
    d = report_dict(rep)
    return {"algo": d["algo"], "n_min": d["n_min"], "depth": d["depth"]}, d


def predict_time(t_sample, m, rows):
    return float(lib().mpgemm_predict_time(float(t_sample), int(m), int(rows)))


def sample_rows(fmt, m, n, n_min, num_sms=152):
    return int(lib().mpgemm_sample_rows(KIND[fmt], int(m), int(n), int(n_min), int(num_sms)))


# ctypes prototype of mpgemm_timer_fn
TIMER_FN = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64,
                            ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.c_int64, ctypes.c_int)


def cache_open(path):
    """Open (or with None close) the persistent tuning cache file."""
    check(lib().mpgemm_tune_cache_open(None if path is None else os.fsencode(path)))


def cache_stats():
    c, mm, s, f = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    is_open = lib().mpgemm_tune_cache_stats(ctypes.byref(c), ctypes.byref(mm), ctypes.byref(s), ctypes.byref(f))
    return {"open": bool(is_open), "choices": c.value, "measurements": mm.value, "skipped_lines": s.value,
            "foreign_records": f.value}


_timer_ref = None


def set_timer(fn):
    """Replace device timing by fn(kind, prec_bits, m, l, n, algo, n_min,
    depth, rows, reps) -> ms (None restores device timing)."""
    global _timer_ref
    if fn is None:
        _timer_ref = None
        check(lib().mpgemm_tune_set_timer(None, None))
        return
    cb = TIMER_FN(lambda ctx, *a: float(fn(*a)))
    _timer_ref = cb
    check(lib().mpgemm_tune_set_timer(ctypes.cast(cb, ctypes.c_void_p), None))


def tune_shape(fmt, m, l, n, flags=REMEMBER, prec_bits=0):
    """mpgemm_tune on placeholder operand pointers, for use with set_timer
    (nothing is launched while a timer is set); returns the report dict."""
    if _timer_ref is None:
        raise RuntimeError("tune_shape needs a timer (set_timer): it passes no operands")
    kind = KIND["mp" if fmt.startswith("mp") else fmt]
    rep = TuneReport()
    fake = ctypes.c_void_p(256)
    check(lib().mpgemm_tune(kind, int(prec_bits), int(m), int(l), int(n), fake, fake, fake, int(flags), None,
                            ctypes.byref(rep)))
    return report_dict(rep)
