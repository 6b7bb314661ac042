"""Error paths under host-side fault injection (mpgemm_fault_inject), on the
GPU: an allocation that fails (Strassen, split-precision and integer-pipe
workspace; every allocation of a batched plan) and a launch check that
reports a failure after a launch that did run (every launch of a Strassen
call).  Each call returns its error, launches nothing after it, leaves the
device status word clear and does not keep its stream-ordered workspace;
the next call without a fault computes the same bits as before.  Nothing is
done to the GPU itself."""

import ctypes

import numpy as np
import pytest

from gpu_util import dev, host
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")

ALLOC, LAUNCH = 1, 2


def _dd(Ad, Bd, Cd, algo=2, n_min=32, depth=2):
    import torch
    m, l, n = Ad.shape[1], Ad.shape[2], Bd.shape[2]
    return mpg.lib().mpgemm_dd(m, l, n, ctypes.c_void_p(Ad.data_ptr()), ctypes.c_void_p(Bd.data_ptr()),
                               ctypes.c_void_p(Cd.data_ptr()), algo, n_min, depth,
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


@pytest.fixture()
def operands():
    import torch
    n = 384
    Ad, Bd = dev(I.dd_random(n, n, 901, 20)), dev(I.dd_random(n, n, 902, 20))
    want = host(mpg.gemm_dd(Ad, Bd, algo="strassen", n_min=32, depth=2))
    yield Ad, Bd, want
    mpg.lib().mpgemm_fault_inject(0, 0)
    torch.cuda.synchronize()


def test_workspace_allocation_fault(operands):
    import torch
    Ad, Bd, want = operands
    L = mpg.lib()
    mpg.set_workspace(None)
    Cd = torch.full_like(Ad, float("nan"))
    fired = L.mpgemm_fault_fired()
    assert L.mpgemm_fault_inject(ALLOC, 0) == 0
    assert _dd(Ad, Bd, Cd) == -6                       # MPGEMM_ENOMEM
    assert L.mpgemm_fault_fired() == fired + 1 and L.mpgemm_last_cuda_error() == 2
    assert mpg.stream_status() == 0
    assert torch.isnan(Cd).all()                       # nothing was launched
    assert _dd(Ad, Bd, Cd) == 0
    assert np.array_equal(host(Cd), want)


def test_launch_fault_at_every_launch_of_a_strassen_call(operands):
    import torch
    Ad, Bd, want = operands
    L = mpg.lib()
    Cd = torch.empty_like(Ad)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # depth 2: two operand launches, the leaf launch, two assembly launches
    for after in range(5):
        assert L.mpgemm_fault_inject(LAUNCH, after) == 0
        assert _dd(Ad, Bd, Cd) == -3, after          # MPGEMM_ECUDA
        assert L.mpgemm_last_cuda_error() == 719
        assert mpg.stream_status() == 0, after       # the launches that ran were sound
    assert L.mpgemm_fault_inject(LAUNCH, 50) == 0 and _dd(Ad, Bd, Cd) == 0   # not reached: no fault
    assert L.mpgemm_fault_inject(0, 0) == 0
    torch.cuda.synchronize()
    # the workspace of every failed call went back on its stream
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
    assert _dd(Ad, Bd, Cd) == 0
    assert np.array_equal(host(Cd), want)


def test_split_precision_and_integer_pipe_allocation_faults(operands):
    import torch
    Ad, Bd, _ = operands
    L = mpg.lib()
    m = Ad.shape[1]
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    Cd = torch.full_like(Ad, float("nan"))
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    want = host(mpg.gemm_split(Ad, Bd, slices=22))
    assert L.mpgemm_fault_inject(ALLOC, 0) == 0
    assert L.mpgemm_dd_ozaki_ex(m, m, m, p(Ad), p(Bd), p(Cd), 22, 1, sp) == -6
    assert torch.isnan(Cd).all()
    assert L.mpgemm_dd_ozaki_ex(m, m, m, p(Ad), p(Bd), p(Cd), 22, 1, sp) == 0
    assert np.array_equal(host(Cd), want)
    want = host(mpg.gemm_via_mp(Ad, Bd, 128, algo="block", n_min=16))
    Cd.fill_(float("nan"))
    assert L.mpgemm_fault_inject(ALLOC, 0) == 0
    with pytest.raises(Exception):
        mpg.gemm_via_mp(Ad, Bd, 128, Cd, algo="block", n_min=16)
    assert torch.isnan(Cd).all()
    assert np.array_equal(host(mpg.gemm_via_mp(Ad, Bd, 128, Cd, algo="block", n_min=16)), want)
    assert mpg.stream_status() == 0


def test_batched_plan_allocation_faults():
    import torch
    from paper_1710_01839_gb300 import batched
    shapes = [("dd", 40, 72, 56), ("qd", 33, 17, 64), ("mp256", 48, 40, 24), ("dd", 100, 30, 70)]
    probs = []
    for i, (fmt, m, l, n) in enumerate(shapes):
        if fmt == "dd":
            A, B, planes, dt = I.dd_random(m, l, 70 + i), I.dd_random(l, n, 80 + i), 2, torch.float64
        elif fmt == "qd":
            A, B, planes, dt = I.qd_random(m, l, 70 + i), I.qd_random(l, n, 80 + i), 4, torch.float64
        else:
            A = I.mp_random(m, l, 8, 70 + i).view(np.int32)
            B = I.mp_random(l, n, 8, 80 + i).view(np.int32)
            planes, dt = 10, torch.int32
        probs.append((fmt, dev(A), dev(B), torch.zeros((planes, m, n), dtype=dt, device="cuda")))
    L = mpg.lib()
    for integer_pipe in (False, True):
        # explicit tiles: with tile 0 the plan would ask the cost model, whose
        # own prediction buffers are allocations that fail gracefully
        descs = batched.make_descs(probs, tiles=[16, 32, 16, 32], integer_pipe=integer_pipe)
        batched.sequential(descs)
        want = [host(c).copy() for _, _, _, c in probs]
        # every allocation the plan makes fails in turn; the plan is not created
        for after in range(6):
            fired = L.mpgemm_fault_fired()
            assert L.mpgemm_fault_inject(ALLOC, after) == 0
            h = ctypes.c_void_p()
            rc = L.mpgemm_batched_plan(descs, len(descs), ctypes.byref(h))
            if L.mpgemm_fault_fired() == fired:          # fewer allocations than `after + 1`
                assert rc == 0
                L.mpgemm_batched_destroy(h)
                break
            assert rc == -6 and not h.value, (integer_pipe, after, rc)
        assert L.mpgemm_fault_inject(0, 0) == 0
        for _, _, _, c in probs:
            c.zero_()
        plan = batched.Plan(descs)
        plan.run_graph()
        plan.close()
        assert mpg.stream_status() == 0
        for (_, _, _, c), w in zip(probs, want):
            assert np.array_equal(host(c), w)
