"""The DD Strassen entry point that allocates nothing
(mpgemm_dd_strassen_noalloc): some callers may not allocate device memory
while they run (their memory is all owned by their own pool allocator, or an
allocation's synchronisation is not acceptable), so this entry point works
on a fixed scratch array inside the library instead.  It runs the same
kernels as the allocating entry point, mpgemm_dd with MPGEMM_STRASSEN, on the
same zero-extended problem, so the two agree bit for bit: checked through the
C ABI on two calls in a row with different inputs (the scratch keeps the
previous call's contents), on an SM partition's stream, and against the
exact product within the Strassen tolerance 2^-96 l max|A| max|B|.  This
file is collected last on purpose."""

import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from gpu_util import dev, host, sample_indices
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _noalloc(Ad, Bd, n_min, depth, stream=None):
    import torch
    m, l, n = Ad.shape[1], Ad.shape[2], Bd.shape[2]
    Cd = torch.full((2, m, n), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    handle = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = mpg.lib().mpgemm_dd_strassen_noalloc(m, l, n, ctypes.c_void_p(Ad.data_ptr()), ctypes.c_void_p(Bd.data_ptr()),
                                              ctypes.c_void_p(Cd.data_ptr()), n_min, depth, ctypes.c_void_p(handle))
    return rc, Cd


def _strassen_bound(A, B):
    l = A.shape[2]
    return 2.0**-96 * l * np.max(np.abs(A[0] + A[1])) * np.max(np.abs(B[0] + B[1]))


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    n, depth, n_min = 256, 2, 32
    for call, seed in enumerate((811, 812)):
        A = I.dd_random(n, n, seed, exp_spread=20)
        B = I.dd_random(n, n, seed + 100, exp_spread=20)
        Ad, Bd = dev(A), dev(B)
        want = host(mpg.gemm_dd(Ad, Bd, algo="strassen", n_min=n_min, depth=depth))
        rc, Cd = _noalloc(Ad, Bd, n_min, depth)
        assert rc == 0, mpg.strerror(rc)
        got = host(Cd)
        assert np.isfinite(got).all(), call
        assert np.array_equal(got, want), call
        ii, jj = sample_indices(n, n, 300, seed=call)
        err, _ = oracle.exact_check(A, B, got, ii, jj)
        assert np.max(err) <= _strassen_bound(A, B), call
    assert mpg.stream_status() == 0


def test_noalloc_refuses_problems_beyond_its_scratch():
    import torch
    n = 1024   # depth 1 needs 7 * 3 * 512^2 * 16 B = 84 MiB > 32 MiB
    Ad = torch.zeros((2, n, n), dtype=torch.float64, device="cuda")
    Bd = torch.zeros((2, n, n), dtype=torch.float64, device="cuda")
    rc, Cd = _noalloc(Ad, Bd, 64, 1)
    assert rc == -6   # MPGEMM_ENOMEM, nothing launched
    torch.cuda.synchronize()
    assert torch.isnan(Cd).all()
    rc, _ = _noalloc(Ad[:, :64, :64].contiguous(), Bd[:, :64, :64].contiguous(), 16, 0)
    assert rc == -1   # depth 0 is not a Strassen call


def test_noalloc_odd_sizes_match_allocating_entry_point():
    """Sizes 2^depth does not divide are zero-extended, here as in mpgemm_dd:
    the same kernels on the same extended problem give the same bits."""
    m, l, n, depth = 253, 255, 257, 2
    A = I.dd_random(m, l, 821, exp_spread=20)
    B = I.dd_random(l, n, 822, exp_spread=20)
    Ad, Bd = dev(A), dev(B)
    want = host(mpg.gemm_dd(Ad, Bd, algo="strassen", n_min=32, depth=depth))
    rc, Cd = _noalloc(Ad, Bd, 32, depth)
    assert rc == 0, mpg.strerror(rc)
    got = host(Cd)
    assert np.array_equal(got, want)
    ii, jj = sample_indices(m, n, 300, seed=5)
    err, _ = oracle.exact_check(A, B, got, ii, jj)
    assert np.max(err) <= _strassen_bound(A, B)


def test_noalloc_on_partition_stream_matches_default_stream():
    """On an SM partition's stream the call runs in the partition's context,
    and gives the bits of the allocating entry point on the default stream."""
    n, depth, n_min = 256, 2, 32
    A = I.dd_random(n, n, 831, exp_spread=20)
    B = I.dd_random(n, n, 832, exp_spread=20)
    Ad, Bd = dev(A), dev(B)
    want = host(mpg.gemm_dd(Ad, Bd, algo="strassen", n_min=n_min, depth=depth))
    with mpg.Partition(24) as p:
        rc, Cd = _noalloc(Ad, Bd, n_min, depth, stream=p.handle)
        assert rc == 0, mpg.strerror(rc)
        assert mpg.stream_status(p.stream) == 0
        assert np.array_equal(host(Cd), want)


_FIRST_ON_PARTITION = r"""
import ctypes, sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
import paper_1710_01839_gb300 as mpg
from paper_1710_01839_gb300 import inputs as I
n, depth, n_min = 128, 1, 32
A = torch.from_numpy(I.dd_random(n, n, 841, exp_spread=20)).cuda()
B = torch.from_numpy(I.dd_random(n, n, 842, exp_spread=20)).cuda()
def call(handle):
    C = torch.full((2, n, n), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    rc = mpg.lib().mpgemm_dd_strassen_noalloc(n, n, n, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                              ctypes.c_void_p(C.data_ptr()), n_min, depth, ctypes.c_void_p(handle))
    assert rc == 0, rc
    return C
p = mpg.Partition(24)
C1 = call(p.handle)            # the library's first call in this process
assert mpg.stream_status(p.stream) == 0
C1 = C1.cpu().numpy()
p.close()                       # the partition's context is gone
C2 = call(torch.cuda.current_stream().cuda_stream)
assert mpg.stream_status() == 0
want = mpg.gemm_dd(A, B, algo="strassen", n_min=n_min, depth=depth).cpu().numpy()
assert np.array_equal(C1, want)
assert np.array_equal(C2.cpu().numpy(), want)
print("ok")
"""


def test_noalloc_first_call_on_partition_then_default_stream():
    """In a fresh process the library's first call comes on a partition's
    stream; after the partition is destroyed a call on the default stream
    still finds the scratch and the status word (both resolved in the
    device's primary context)."""
    env = dict(os.environ)
    r = subprocess.run([sys.executable, "-c", _FIRST_ON_PARTITION.format(root=ROOT)], capture_output=True,
                       text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert r.stdout.strip().endswith("ok")
