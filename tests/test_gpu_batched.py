"""Batched uneven mixed-precision GEMMs in one persistent launch: results are
bit-identical to one ordinary block launch per GEMM (same tile code, same
per-element operation order), identical across graph replays, and agree with
the oracle (DD bound, multi-limb bit-exact)."""

import numpy as np
import pytest

import oracle
from gpu_util import DD_BOUND, QD_BOUND, bound_ratio, dev, host
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")


def _problems(shapes, seed):
    import torch
    probs, hostdata = [], []
    for i, (m, l, n, prec) in enumerate(shapes):
        s = seed + 7 * i
        if prec == "dd":
            A, B = I.dd_random(m, l, s), I.dd_random(l, n, s + 1)
            C = torch.empty((2, m, n), dtype=torch.float64, device="cuda")
        elif prec == "qd":
            A, B = I.qd_random(m, l, s), I.qd_random(l, n, s + 1)
            C = torch.empty((4, m, n), dtype=torch.float64, device="cuda")
        else:
            A, B = I.mp_random(m, l, 8, s), I.mp_random(l, n, 8, s + 1)
            C = torch.empty((10, m, n), dtype=torch.int32, device="cuda")
        probs.append((prec, dev(A), dev(B), C))
        hostdata.append((A, B))
    return probs, hostdata


def _snapshot(probs):
    return [host(C, mp=(p == "mp256")).copy() for p, _, _, C in probs]


def test_persistent_equals_sequential_and_graph():
    from paper_1710_01839_gb300 import batched
    rng = np.random.default_rng(5)
    shapes = [(int(rng.integers(1, 150)), int(rng.integers(0, 150)), int(rng.integers(1, 150)),
               ["dd", "qd", "mp256"][i % 3]) for i in range(36)]
    shapes += [(33, 1, 17, "dd"), (1, 1, 1, "qd"), (16, 16, 16, "mp256"), (64, 0, 5, "mp256")]
    probs, hostdata = _problems(shapes, 100)
    tiles = [16 if i % 2 else 32 for i in range(len(probs))]
    descs = batched.make_descs(probs, tiles)
    batched.sequential(descs)
    ref = _snapshot(probs)
    for _, _, _, C in probs:
        C.zero_()
    plan = batched.Plan(descs)
    info = plan.info()
    assert info["grid"] >= 152 and info["work_items"] > 0
    plan.run()
    got = _snapshot(probs)
    for r, g in zip(ref, got):
        assert np.array_equal(r, g)
    for rep in range(2):
        for _, _, _, C in probs:
            C.zero_()
        plan.run_graph()
        for r, g in zip(ref, _snapshot(probs)):
            assert np.array_equal(r, g), rep
    plan.close()
    assert mpg.stream_status() == 0
    # against the oracle
    for (prec, _, _, _), (A, B), C in zip(probs, hostdata, got):
        m, n = C.shape[1], C.shape[2]
        if A.shape[2] == 0:
            if prec == "mp256":
                assert (C[1] == 2).all()
            else:
                assert not C.any()
            continue
        if prec == "mp256":
            assert np.array_equal(C, oracle.mp_gemm(A, B, prec_bits=256))
        else:
            ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
            rel = DD_BOUND if prec == "dd" else QD_BOUND
            assert bound_ratio(A, B, C, ii.ravel().astype(np.int64), jj.ravel().astype(np.int64), rel) <= 1.0


def test_config_workload_persistent_matches_sequential():
    # the 512-GEMM uneven workload's first 96 GEMMs (sizes log-uniform in [16, 1024])
    from paper_1710_01839_gb300 import batched
    shapes = I.batched_shapes()[:96]
    probs, _ = _problems(shapes, 2000)
    descs = batched.make_descs(probs)
    batched.sequential(descs)
    ref = _snapshot(probs)
    plan = batched.Plan(descs)
    plan.run_graph()
    for r, g in zip(ref, _snapshot(probs)):
        assert np.array_equal(r, g)
    plan.close()


def test_plan_rejects_bad_descriptors():
    import ctypes
    from paper_1710_01839_gb300 import batched
    import torch
    A = torch.zeros((10, 4, 4), dtype=torch.int32, device="cuda")
    d = batched.make_descs([("mp256", A, A, A)])
    d[0].prec_bits = 128          # the batched kernel only carries 256-bit multi-limb
    h = ctypes.c_void_p()
    assert mpg.lib().mpgemm_batched_plan(d, 1, ctypes.byref(h)) == -2
    d[0].prec_bits = 256
    d[0].m = -1
    assert mpg.lib().mpgemm_batched_plan(d, 1, ctypes.byref(h)) == -1


def test_integer_pipe_engine_equals_sequential_graph_and_oracle():
    # DD and QD descriptors with engine = 1 (128 / 256-bit limbs, conversion
    # passes around the persistent kernel) beside ordinary 256-bit ones:
    # persistent == graph replay == one mpgemm_*_via_mp launch per GEMM ==
    # the oracle's conversion + multi-limb GEMM, bit for bit
    from paper_1710_01839_gb300 import batched
    rng = np.random.default_rng(9)
    shapes = [(int(rng.integers(1, 90)), int(rng.integers(0, 90)), int(rng.integers(1, 90)),
               ["dd", "qd", "mp256"][i % 3]) for i in range(24)]
    shapes += [(40, 1, 23, "dd"), (1, 1, 1, "qd"), (17, 0, 9, "dd")]
    probs, hostdata = _problems(shapes, 300)
    descs = batched.make_descs(probs, integer_pipe=True)
    assert [d.engine for d in descs] == [0 if p == "mp256" else 1 for p, _, _, _ in probs]
    batched.sequential(descs)
    ref = _snapshot(probs)
    plan = batched.Plan(descs)
    assert set(plan.info()["tiles"]) == {16}
    for _, _, _, C in probs:
        C.zero_()
    plan.run()
    got = _snapshot(probs)
    for r, g in zip(ref, got):
        assert np.array_equal(r.view(np.uint8), g.view(np.uint8))
    for _ in range(2):
        for _, _, _, C in probs:
            C.zero_()
        plan.run_graph()
        for r, g in zip(ref, _snapshot(probs)):
            assert np.array_equal(r.view(np.uint8), g.view(np.uint8))
    plan.close()
    assert mpg.stream_status() == 0
    for (prec, _, _, _), (A, B), C in zip(probs, hostdata, got):
        if prec == "mp256":
            assert np.array_equal(C, oracle.mp_gemm(A, B, prec_bits=256))
        elif A.shape[2] == 0:
            assert not C.any()
        else:
            bits = 128 if prec == "dd" else 256
            Co = oracle.gemm_via_mp(A, B, bits, algo="block", n_min=16)
            assert np.array_equal(C.view(np.uint64), Co.view(np.uint64))


def test_plan_rejects_bad_engine():
    import ctypes
    from paper_1710_01839_gb300 import batched
    import torch
    A = torch.zeros((6 + 4, 4, 4), dtype=torch.int32, device="cuda")
    D = torch.zeros((2, 4, 4), dtype=torch.float64, device="cuda")
    h = ctypes.c_void_p()
    d = batched.make_descs([("mp256", A, A, A)])
    d[0].engine = 1               # the integer pipe is for DD / QD descriptors
    assert mpg.lib().mpgemm_batched_plan(d, 1, ctypes.byref(h)) == -1
    d = batched.make_descs([("dd", D, D, D)])
    d[0].engine = 2
    assert mpg.lib().mpgemm_batched_plan(d, 1, ctypes.byref(h)) == -1


def test_mixed_engines_in_one_plan():
    # engine 0 and engine 1 descriptors of the same formats in one plan: the
    # full persistent kernel runs FP64 DD / QD tiles beside 128- and 256-bit
    # ones; each result equals its own engine's sequential launch
    from paper_1710_01839_gb300 import batched
    shapes = [(37, 29, 23, "dd"), (40, 33, 17, "qd"), (25, 31, 19, "dd"), (18, 26, 30, "qd"), (20, 20, 20, "mp256")]
    probs, _ = _problems(shapes, 500)
    descs = batched.make_descs(probs, [32] * len(probs))
    for i, d in enumerate(descs):
        if i in (2, 3):
            d.engine = 1
    batched.sequential(descs)
    ref = _snapshot(probs)
    for _, _, _, C in probs:
        C.zero_()
    plan = batched.Plan(descs)
    assert plan.info()["tiles"] == [32, 32, 16, 16, 16]
    plan.run_graph()
    for r, g in zip(ref, _snapshot(probs)):
        assert np.array_equal(r.view(np.uint8), g.view(np.uint8))
    plan.close()
    assert mpg.stream_status() == 0
