"""Device failure path: every wait in the library's kernels is bounded, and a
wait that runs out is reported, not hung.  The self-test runs the kernels'
own bounded mbarrier wait on a phase that nothing ever completes (no fault,
no trap, nothing left running); the host must read MPGEMM_ETIMEOUT, the
status word must be cleared, and the context must stay usable."""

import ctypes
import time

import numpy as np
import pytest

import oracle
from gpu_util import dev, host
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")


def _sp():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("limit_ms", [20, 200])
def test_bounded_wait_reports_timeout_and_context_survives(limit_ms):
    L = mpg.lib()
    t0 = time.perf_counter()
    assert L.mpgemm_selftest_wait_timeout(limit_ms, _sp()) == -5      # MPGEMM_ETIMEOUT
    elapsed = time.perf_counter() - t0
    assert limit_ms / 1e3 * 0.9 <= elapsed < limit_ms / 1e3 + 5.0      # it waited, then gave up
    assert mpg.stream_status() == 0                                    # the status word was cleared
    A, B = I.dd_random(33, 21, 5), I.dd_random(21, 17, 6)
    C = host(mpg.gemm_dd(dev(A), dev(B), algo="block"))                # the context still works
    assert np.array_equal(C, host(mpg.gemm_dd(dev(A), dev(B), algo="simple")))
    ii, jj = np.meshgrid(np.arange(33), np.arange(17), indexing="ij")
    err, absab = oracle.exact_check(A, B, C, ii.ravel(), jj.ravel())
    assert np.all(err <= 4 * 21 * 2.0**-104 * absab)


def test_timeout_on_a_partition_stream():
    with mpg.Partition(24) as p:
        assert mpg.lib().mpgemm_selftest_wait_timeout(20, ctypes.c_void_p(p.handle)) == -5
        assert mpg.stream_status(p.stream) == 0
