"""SM partitions (green contexts), the GPU counterpart of the paper's thread
counts: the same kernels on a subset of the SMs give bit-identical results,
the library sizes its work by the partition's SM count (the persistent
tcgen05 grid, the tuner's rounds model), the tuner's predictions stay within
the paper's 10 % on a partition, and a partition really runs on fewer SMs."""

import ctypes

import numpy as np
import pytest

from gpu_util import dev, host
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")


def _device_sms():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


def test_partition_block_gemm_bit_identical():
    import torch
    A, B = I.dd_random(300, 200, 31, 20), I.dd_random(200, 170, 32, 20)
    Ad, Bd = dev(A), dev(B)
    full = host(mpg.gemm_dd(Ad, Bd, algo="block", n_min=32))
    torch.cuda.synchronize()
    with mpg.Partition(38) as p:
        assert 38 <= p.sms < _device_sms()
        assert mpg.lib().mpgemm_stream_sms(ctypes.c_void_p(p.handle)) == p.sms
        C = mpg.gemm_dd(Ad, Bd, algo="block", n_min=32, stream=p.stream)
        assert mpg.stream_status(p.stream) == 0
        assert np.array_equal(host(C), full)
        # the default stream still reports the whole device
        assert mpg.lib().mpgemm_stream_sms(None) == _device_sms()


def test_partition_fp8_split_precision_bit_identical():
    import torch
    m, l, n = 520, 300, 530
    A, B = I.dd_rowcol_scaled(m, l, n, seed=41)
    Ad, Bd = dev(A), dev(B)
    C0 = torch.empty((2, m, n), dtype=torch.float64, device="cuda")
    C1 = torch.empty_like(C0)
    L = mpg.lib()
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.mpgemm_dd_ozaki_ex(m, l, n, ctypes.c_void_p(Ad.data_ptr()), ctypes.c_void_p(Bd.data_ptr()),
                                ctypes.c_void_p(C0.data_ptr()), 22, 1, sp) == 0
    torch.cuda.synchronize()
    with mpg.Partition(24) as p:
        assert L.mpgemm_dd_ozaki_ex(m, l, n, ctypes.c_void_p(Ad.data_ptr()), ctypes.c_void_p(Bd.data_ptr()),
                                    ctypes.c_void_p(C1.data_ptr()), 22, 1, ctypes.c_void_p(p.handle)) == 0
        assert mpg.stream_status(p.stream) == 0
    assert np.array_equal(host(C1), host(C0))


def test_partition_tuner_predicts_and_runs_slower():
    from paper_1710_01839_gb300 import tuner
    import torch
    n = 1024
    A, B = I.dd_random(n, n, 51, 20), I.dd_random(n, n, 52, 20)
    Ad, Bd = dev(A), dev(B)
    Cd = torch.empty_like(Ad)
    _, full = tuner.tune("dd", Ad, Bd, Cd, flags=tuner.VERIFY | tuner.SKIP_SIMPLE | tuner.QUICK)
    torch.cuda.synchronize()
    with mpg.Partition(38) as p:
        _, part = tuner.tune("dd", Ad, Bd, Cd, flags=tuner.VERIFY | tuner.SKIP_SIMPLE | tuner.QUICK,
                             stream=p.stream)
    assert part["max_prediction_rel_diff"] <= 0.10
    # a quarter of the SMs: the block GEMM takes well over twice as long
    assert part["block_ms"] > 2.0 * full["block_ms"]


def test_partition_arguments():
    L = mpg.lib()
    h, k = ctypes.c_void_p(), ctypes.c_int()
    assert L.mpgemm_partition_create(0, ctypes.byref(h), ctypes.byref(k)) == -1
    assert L.mpgemm_partition_create(100000, ctypes.byref(h), ctypes.byref(k)) == -1
    assert L.mpgemm_partition_destroy(ctypes.c_void_p(12345)) == -1
