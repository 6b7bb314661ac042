"""The DD Strassen entry point that allocates nothing
(mpgemm_dd_strassen_noalloc): some callers may not allocate device memory
while they run (their memory is all owned by their own pool allocator, or an
allocation's synchronisation is not acceptable), so this entry point works
on a fixed scratch array inside the library instead.  Checked through the
C ABI against the allocating entry point, mpgemm_dd with MPGEMM_STRASSEN, on
two calls in a row with different inputs (the scratch keeps the previous
call's contents), within the Strassen tolerance the other tests use,
2^-96 l max|A| max|B|.  This file is collected last on purpose."""

import ctypes

import numpy as np
import pytest

from gpu_util import dev, host
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")


def _noalloc(Ad, Bd, n_min, depth):
    import torch
    m, l, n = Ad.shape[1], Ad.shape[2], Bd.shape[2]
    Cd = torch.full((2, m, n), float("nan"), dtype=torch.float64, device="cuda")
    rc = mpg.lib().mpgemm_dd_strassen_noalloc(m, l, n, ctypes.c_void_p(Ad.data_ptr()), ctypes.c_void_p(Bd.data_ptr()),
                                              ctypes.c_void_p(Cd.data_ptr()), n_min, depth,
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, Cd


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
        tol = 2.0**-96 * n * np.max(np.abs(A[0])) * np.max(np.abs(B[0]))
        diff = np.abs((got[0] - want[0]) + (got[1] - want[1]))
        assert np.max(diff) <= tol, (call, float(np.max(diff)), tol)
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
    assert np.array_equal(host(Cd), want)
