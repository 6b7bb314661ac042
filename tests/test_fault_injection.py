"""Host-side fault injection (mpgemm_fault_inject, MPGEMM_FAULT) without a
GPU: argument checks, and an armed allocation fault reaching the Strassen
workspace allocation (a path that needs no CUDA call before it), both from
the API and from the environment variable.  The GPU-side error paths are in
test_gpu_fault_injection.py."""

import ctypes
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1710_01839_gb300 import build
    build.build()
    import paper_1710_01839_gb300 as mpg
    return mpg.lib()


def test_arguments(L):
    assert L.mpgemm_fault_inject(3, 0) == -1
    assert L.mpgemm_fault_inject(1, -1) == -1
    assert L.mpgemm_fault_inject(0, 0) == 0


_CHILD = r"""
import ctypes, sys
sys.path.insert(0, {root!r})
import paper_1710_01839_gb300 as mpg
L = mpg.lib()
p = ctypes.c_void_p(4096)
q = ctypes.c_void_p(1 << 40)
{arm}
out = []
for _ in range(2):
    rc = L.mpgemm_dd(64, 64, 64, p, ctypes.c_void_p(1 << 30), q, 2, 16, 1, None)   # MPGEMM_STRASSEN, depth 1
    out.append((rc, L.mpgemm_fault_fired(), L.mpgemm_last_cuda_error()))
print(out)
"""


def _child(arm, env_fault=None):
    env = dict(os.environ)
    env.pop("MPGEMM_FAULT", None)
    if env_fault:
        env["MPGEMM_FAULT"] = env_fault
    env["CUDA_VISIBLE_DEVICES"] = ""   # the same on a GPU machine: no device call is reached before the fault
    r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT, arm=arm)], capture_output=True, text=True,
                       timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    return eval(r.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("how", ["api", "env"])
def test_allocation_fault_reaches_the_workspace(L, how):
    if how == "api":
        res = _child("assert L.mpgemm_fault_inject(1, 1) == 0")
    else:
        res = _child("", env_fault="alloc:1")
    # first call: the fault counts down (1 -> 0) and the allocation proceeds to
    # the device, which is not there; second call: the fault fires
    (rc1, fired1, _), (rc2, fired2, err2) = res
    assert rc1 == -3 and fired1 == 0
    assert rc2 == -6 and fired2 == 1 and err2 == 2    # MPGEMM_ENOMEM, cudaErrorMemoryAllocation


def test_malformed_environment_is_ignored(L):
    (rc1, fired1, _), (rc2, fired2, _) = _child("", env_fault="alloc:x")
    assert fired1 == fired2 == 0 and rc1 == rc2 == -3
