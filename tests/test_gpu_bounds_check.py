"""The bounds-checked build (libmpgemm_bc.so: the library's sources compiled
with -DMPGEMM_BOUNDS_CHECK): every global read and write of the DD, QD and
multi-limb simple, block and Strassen kernels is checked against the buffer
it belongs to, an access outside is not made and is counted
(mpgemm_bounds_read).  Its self-test counts exactly its two planted misses
(both stay inside a larger allocation, so nothing outside any allocation is
touched even without the check); then every algorithm, at sizes that are
multiples of no tile (1 x 1 x 1, primes, ragged; Strassen's zero extension
at depths 1-4), the one-thread and the warp-cooperative multi-limb kernels
and DD / QD on the integer pipe make no access outside their buffers and
give the same bits as the normal build."""

import ctypes

import numpy as np
import pytest

from gpu_util import host
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")

SHAPES = [(1, 1, 1), (2, 3, 5), (17, 31, 13), (37, 53, 29), (65, 33, 47)]
CONFIGS = [(0, 16, 0), (1, 16, 0), (1, 32, 0), (1, 64, 0), (2, 16, 1), (2, 16, 2), (2, 16, 3), (2, 16, 4)]


@pytest.fixture(scope="module")
def Lc():
    from paper_1710_01839_gb300._lib import lib_checked
    return lib_checked()


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _misses(Lc):
    count, first = ctypes.c_longlong(), ctypes.c_ulonglong()
    assert Lc.mpgemm_bounds_read(ctypes.byref(count), ctypes.byref(first)) == 0
    return count.value, first.value


def test_selftest_counts_the_planted_misses(Lc):
    _misses(Lc)
    assert Lc.mpgemm_selftest_bounds(_stream()) == 0
    count, first = _misses(Lc)
    assert count == 2 and first != 0
    assert _misses(Lc) == (0, 0)           # read clears
    assert mpg.lib().mpgemm_bounds_read(None, None) == -2      # the normal build has no counter


@pytest.mark.parametrize("fmt", ["dd", "qd"])
def test_dd_qd_no_access_outside(Lc, fmt):
    import torch
    P = 2 if fmt == "dd" else 4
    gen = I.dd_random if fmt == "dd" else I.qd_random
    fn = Lc.mpgemm_dd if fmt == "dd" else Lc.mpgemm_qd
    ref = mpg.gemm_dd if fmt == "dd" else mpg.gemm_qd
    _misses(Lc)
    for m, l, n in SHAPES:
        A = torch.from_numpy(gen(m, l, 31 + m, exp_spread=20)).cuda()
        B = torch.from_numpy(gen(l, n, 32 + n, exp_spread=20)).cuda()
        for algo, nm, d in CONFIGS:
            C = torch.full((P, m, n), float("nan"), dtype=torch.float64, device="cuda")
            assert fn(m, l, n, _p(A), _p(B), _p(C), algo, nm, d, _stream()) == 0
            want = host(ref(A, B, algo=["simple", "block", "strassen"][algo], n_min=nm, depth=d))
            assert np.array_equal(host(C), want), (m, l, n, algo, nm, d)
        assert _misses(Lc) == (0, 0), (m, l, n)


@pytest.mark.parametrize("w,leaf", [(1, 1), (4, 1), (8, 1), (16, 1), (32, 1), (64, 1), (16, 2), (32, 2), (64, 2)])
def test_multi_limb_no_access_outside(Lc, w, leaf):
    # leaf 1: one thread per output; 2: the warp-cooperative kernel (512-2048 bits)
    import torch
    prev = Lc.mpgemm_set_mp_leaf(leaf)
    prev_n = mpg.set_mp_leaf("thread" if leaf == 1 else "team")
    try:
        _misses(Lc)
        for m, l, n in SHAPES[:4] if w == 64 else SHAPES:
            A = torch.from_numpy(I.mp_random(m, l, w, 41 + m).view(np.int32)).cuda()
            B = torch.from_numpy(I.mp_random(l, n, w, 42 + n).view(np.int32)).cuda()
            for algo, nm, d in CONFIGS:
                C = torch.full((2 + w, m, n), 0x7FC5A5A5, dtype=torch.int32, device="cuda")
                assert Lc.mpgemm_mp(m, l, n, 32 * w, _p(A), _p(B), _p(C), algo, nm, d, _stream()) == 0
                want = host(mpg.gemm_mp(A, B, 32 * w, algo=["simple", "block", "strassen"][algo], n_min=nm, depth=d),
                            mp=True)
                assert np.array_equal(host(C, mp=True), want), (m, l, n, algo, nm, d)
            assert _misses(Lc) == (0, 0), (w, m, l, n)
    finally:
        Lc.mpgemm_set_mp_leaf(prev)
        mpg.set_mp_leaf(prev_n)


@pytest.mark.parametrize("fmt,bits", [("dd", 128), ("qd", 256)])
def test_integer_pipe_no_access_outside(Lc, fmt, bits):
    import torch
    P = 2 if fmt == "dd" else 4
    gen = I.dd_random if fmt == "dd" else I.qd_random
    fn = Lc.mpgemm_dd_via_mp if fmt == "dd" else Lc.mpgemm_qd_via_mp
    _misses(Lc)
    for m, l, n in SHAPES:
        A = torch.from_numpy(gen(m, l, 51 + m, exp_spread=20)).cuda()
        B = torch.from_numpy(gen(l, n, 52 + n, exp_spread=20)).cuda()
        for algo, nm, d in [(1, 16, 0), (2, 16, 2)]:
            C = torch.full((P, m, n), float("nan"), dtype=torch.float64, device="cuda")
            assert fn(m, l, n, _p(A), _p(B), _p(C), bits, algo, nm, d, _stream()) == 0
            want = host(mpg.gemm_via_mp(A, B, bits, algo=["simple", "block", "strassen"][algo], n_min=nm, depth=d))
            assert np.array_equal(host(C), want), (m, l, n, algo)
        assert _misses(Lc) == (0, 0), (m, l, n)
