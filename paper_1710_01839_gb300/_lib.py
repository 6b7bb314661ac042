"""ctypes declarations of libmpgemm's C ABI (include/mpgemm.h)."""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libmpgemm.so")
_LIB_CHECKED_PATH = os.path.join(_HERE, "_build_bc", "libmpgemm_bc.so")

ALGO = {"simple": 0, "block": 1, "strassen": 2, "auto": 3}
KIND = {"dd": 0, "qd": 1, "mp": 2}
STATUS = {0: "MPGEMM_OK", -1: "MPGEMM_EINVAL", -2: "MPGEMM_EUNSUPPORTED", -3: "MPGEMM_ECUDA",
          -4: "MPGEMM_EOVERFLOW", -5: "MPGEMM_ETIMEOUT", -6: "MPGEMM_ENOMEM"}


class MpgemmError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {msg}")


_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_SZ = ctypes.c_size_t

# name -> (restype, argtypes); every function the header declares
SIGNATURES = {
    "mpgemm_dd": (_I, [_I64, _I64, _I64, _P, _P, _P, _I, _I, _I, _P]),
    "mpgemm_qd": (_I, [_I64, _I64, _I64, _P, _P, _P, _I, _I, _I, _P]),
    "mpgemm_mp": (_I, [_I64, _I64, _I64, _I, _P, _P, _P, _I, _I, _I, _P]),
    "mpgemm_workspace_size": (_SZ, [_I, _I, _I64, _I64, _I64, _I, _I]),
    "mpgemm_set_workspace": (_I, [_P, _SZ]),
    "mpgemm_stream_status": (_I, [_P]),
    "mpgemm_selftest_wait_timeout": (_I, [_I, _P]),
    "mpgemm_fault_inject": (_I, [_I, ctypes.c_longlong]),
    "mpgemm_fault_fired": (_I, []),
    "mpgemm_partition_create": (_I, [_I, _P, _P]),
    "mpgemm_precision_log2_bound": (ctypes.c_double, [_I, _I, _I, _I64, _I]),
    "mpgemm_select_precision": (_I, [ctypes.c_double, _I64, _I64, _I64, _I, _P, _I]),
    "mpgemm_dd_exponent_spread": (_I, [_I64, _I64, _I64, _P, _P, _P, _P]),
    "mpgemm_partition_destroy": (_I, [_P]),
    "mpgemm_stream_sms": (_I, [_P]),
    "mpgemm_strerror": (ctypes.c_char_p, [_I]),
    "mpgemm_last_cuda_error": (_I, []),
    "mpgemm_version": (_I, []),
    "mpgemm_peak_run": (_I, [_I, _I64, _P, _P]),
    "mpgemm_profile": (_I, [_I]),
    "mpgemm_cost_num_features": (_I, []),
    "mpgemm_cost_choice": (_I, [_I, _I, _I64, _I64, _I64, _P, _P, _P, _P, _P]),
    "mpgemm_cost_features": (_I, [_I, _I, _I64, _I64, _I64, _I, _I, _I, _P]),
    "mpgemm_cost_collect": (_I, [_I, ctypes.c_ulonglong, _I, _P, _P, _P]),
    "mpgemm_cost_train": (_I, [_P, _P, _I, _I, ctypes.c_ulonglong, _P]),
    "mpgemm_cost_predict": (_I, [_P, _I, _P]),
    "mpgemm_cost_save": (_I, [ctypes.c_char_p]),
    "mpgemm_cost_load": (_I, [ctypes.c_char_p]),
    "mpgemm_cost_clear": (_I, []),
    "mpgemm_batched_plan": (_I, [_P, _I, _P]),
    "mpgemm_batched_run": (_I, [_P, _P]),
    "mpgemm_batched_run_graph": (_I, [_P, _P]),
    "mpgemm_batched_destroy": (_I, [_P]),
    "mpgemm_batched_info": (_I, [_P, _P, _P, _P, _I]),
    "mpgemm_batched_sequential": (_I, [_P, _I, _P]),
    "mpgemm_dd_strassen_noalloc": (_I, [_I64, _I64, _I64, _P, _P, _P, _I, _I, _P]),
    "mpgemm_dd_ozaki": (_I, [_I64, _I64, _I64, _P, _P, _P, _I, _P]),
    "mpgemm_dd_ozaki_ex": (_I, [_I64, _I64, _I64, _P, _P, _P, _I, _I, _P]),
    "mpgemm_ozaki_split_ex": (_I, [_I, _I, _I64, _I64, _P, _I, _P, _P, _P]),
    "mpgemm_ozaki_levels_ex": (_I, [_I, _I64, _I64, _I64, _I, _P, _P, _P, _P]),
    "mpgemm_ozaki_workspace_size": (_SZ, [_I64, _I64, _I64, _I]),
    "mpgemm_ozaki_slices_default": (_I, []),
    "mpgemm_ozaki_split": (_I, [_I, _I64, _I64, _P, _I, _P, _P, _P]),
    "mpgemm_ozaki_levels": (_I, [_I64, _I64, _I64, _I, _P, _P, _P, _P]),
    "mpgemm_qd_ozaki": (_I, [_I64, _I64, _I64, _P, _P, _P, _I, _P]),
    "mpgemm_qd_ozaki_slices_default": (_I, []),
    "mpgemm_split_job_order": (_I, [_I64, _I64, _I64, _I, _P, _I]),
    "mpgemm_ozaki_split_terms": (_I, [_I, _I, _I64, _I64, _P, _I, _P, _P, _P]),
    "mpgemm_tune": (_I, [_I, _I, _I64, _I64, _I64, _P, _P, _P, _I, _P, _P]),
    "mpgemm_tune_forget": (_I, []),
    "mpgemm_auto_mode": (_I, [_I]),
    "mpgemm_set_mp_leaf": (_I, [_I]),
    "mpgemm_bounds_read": (_I, [_P, _P]),
    "mpgemm_selftest_bounds": (_I, [_P]),
    "mpgemm_mp_leaf_choice": (_I, [_I, _I64, _I64, _I64, _I]),
    "mpgemm_time_config": (_I, [_I, _I, _I64, _I64, _I64, _P, _P, _P, _I, _I, _I, _I, _P, _P]),
    "mpgemm_tune_cache_open": (_I, [ctypes.c_char_p]),
    "mpgemm_tune_cache_stats": (_I, [_P, _P, _P, _P]),
    "mpgemm_tune_set_timer": (_I, [_P, _P]),
    "mpgemm_auto_choice": (_I, [_I, _I, _I64, _I64, _I64, _P, _P, _P]),
    "mpgemm_predict_time": (ctypes.c_double, [ctypes.c_double, _I64, _I64]),
    "mpgemm_sample_rows": (_I64, [_I, _I64, _I64, _I, _I]),
    "mpgemm_profile_read": (_I, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "mpgemm_dd_via_mp": (_I, [_I64, _I64, _I64, _P, _P, _P, _I, _I, _I, _I, _P]),
    "mpgemm_qd_via_mp": (_I, [_I64, _I64, _I64, _P, _P, _P, _I, _I, _I, _I, _P]),
    "mpgemm_via_mp_workspace_size": (_SZ, [_I, _I64, _I64, _I64, _I, _I]),
    "mpgemm_terms_to_mp": (_I, [_I, _I64, _P, _I, _P, _P]),
    "mpgemm_mp_to_terms": (_I, [_I, _I64, _I, _P, _P, _P]),
    "mpgemm_selftest_two_sum": (_I, [_I64, _P, _P, _P, _P]),
    "mpgemm_selftest_two_prod": (_I, [_I64, _P, _P, _P, _P]),
    "mpgemm_selftest_dd_mac": (_I, [_I64, _P, _P, _P]),
    "mpgemm_selftest_dd_add": (_I, [_I64, _P, _P, _P]),
}


def lib_path() -> str:
    return _LIB_PATH


def _load(path):
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; "
                           f"g.build()'` (the CUDA library is required; there is no CPU path)")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib():
    """Load libmpgemm.so.  Raises if it was not built (no fallback)."""
    global _lib
    if _lib is None:
        _lib = _load(_LIB_PATH)
    return _lib


_lib_checked = None


def lib_checked():
    """Load the bounds-checked build, libmpgemm_bc.so (a testing tool: the
    same C ABI, every global access of the GEMM kernels checked against its
    buffer; see mpgemm_bounds_read).  It is a separate library with its own
    state (workspace, status word, tuner)."""
    global _lib_checked
    if _lib_checked is None:
        _lib_checked = _load(_LIB_CHECKED_PATH)
    return _lib_checked


def check_planes(t, planes, dtypes, name, rows=None, cols=None):
    """Refuse anything but a contiguous tensor of shape (planes, rows, cols)
    and one of `dtypes` (structure only; require_cuda checks the device once
    every operand's structure has passed, so that each mistake is reported
    as what it is)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype not in dtypes:
        raise TypeError(f"{name} has dtype {t.dtype}, expected one of {dtypes}")
    if t.dim() != 3 or t.shape[0] != planes:
        raise ValueError(f"{name} must have shape ({planes}, rows, cols), got {tuple(t.shape)}")
    if (rows is not None and t.shape[1] != rows) or (cols is not None and t.shape[2] != cols):
        raise ValueError(f"{name} must have shape ({planes}, {rows}, {cols}), got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def require_cuda(**tensors):
    """Every tensor on the same CUDA device (the library has no CPU path)."""
    dev = None
    for name, t in tensors.items():
        if not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor (the library has no CPU path)")
        if dev is not None and t.device != dev:
            raise ValueError(f"{name} is on {t.device}, the other operands on {dev}")
        dev = t.device


def int_dtypes():
    import torch
    return (torch.int32, torch.uint32) if hasattr(torch, "uint32") else (torch.int32,)


def check(rc: int):
    if rc != 0:
        extra = ""
        if rc == -3:
            extra = f"cudaError {lib().mpgemm_last_cuda_error()}"
        raise MpgemmError(rc, lib().mpgemm_strerror(rc).decode() + (" " + extra if extra else ""))
