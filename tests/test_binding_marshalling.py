"""The Python binding hands the C ABI the right sizes, pointers and codes
(no GPU).

The library and the device check are replaced by recorders, so that host
tensors of the right structure go through every entry point; each test then
compares the recorded call with the ABI's argument order in
include/mpgemm.h."""

import ctypes

import pytest

torch = pytest.importorskip("torch")
mpg = pytest.importorskip("paper_1710_01839_gb300")
from paper_1710_01839_gb300 import batched, tuner  # noqa: E402

f64, i32 = torch.float64, torch.int32


class Recorder:
    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        def f(*args):
            self.calls.append((name, args))
            return 0
        return f


def _v(x):
    return x.value if isinstance(x, ctypes.c_void_p) else x


@pytest.fixture
def rec(monkeypatch):
    r = Recorder()
    for mod in (mpg, tuner, batched):
        monkeypatch.setattr(mod, "lib", lambda r=r: r)
        monkeypatch.setattr(mod, "require_cuda", lambda **kw: None)
    monkeypatch.setattr(mpg, "_stream_ptr", lambda stream: ctypes.c_void_p(1234))
    return r


def T(planes, r, c, dtype=f64):
    return torch.zeros((planes, r, c), dtype=dtype)


def test_gemm_dd_qd_mp(rec):
    A, B = T(2, 5, 3), T(2, 3, 4)
    C = mpg.gemm_dd(A, B, algo="strassen", n_min=32, depth=2)
    assert C.shape == (2, 5, 4)
    name, a = rec.calls[-1]
    assert name == "mpgemm_dd"
    assert [_v(x) for x in a] == [5, 3, 4, A.data_ptr(), B.data_ptr(), C.data_ptr(), 2, 32, 2, 1234]
    A4, B4, C4 = T(4, 5, 3), T(4, 3, 4), T(4, 5, 4)
    mpg.gemm_qd(A4, B4, C4, algo="simple")
    name, a = rec.calls[-1]
    assert name == "mpgemm_qd" and [_v(x) for x in a[:7]] == [5, 3, 4, A4.data_ptr(), B4.data_ptr(), C4.data_ptr(), 0]
    Am, Bm = T(6, 5, 3, i32), T(6, 3, 4, i32)
    Cm = mpg.gemm_mp(Am, Bm, 128, algo="auto")
    name, a = rec.calls[-1]
    assert name == "mpgemm_mp" and Cm.shape == (6, 5, 4) and Cm.dtype == i32
    assert [_v(x) for x in a[:8]] == [5, 3, 4, 128, Am.data_ptr(), Bm.data_ptr(), Cm.data_ptr(), 3]


def test_integer_pipe_and_conversions(rec):
    A, B = T(2, 5, 3), T(2, 3, 4)
    C = mpg.gemm_via_mp(A, B)
    name, a = rec.calls[-1]
    assert name == "mpgemm_dd_via_mp"
    assert [_v(x) for x in a[:8]] == [5, 3, 4, A.data_ptr(), B.data_ptr(), C.data_ptr(), 128, 1]
    A4, B4 = T(4, 5, 3), T(4, 3, 4)
    C4 = mpg.gemm_via_mp(A4, B4, algo="strassen", n_min=16, depth=1)
    name, a = rec.calls[-1]
    assert name == "mpgemm_qd_via_mp" and [_v(x) for x in a[6:10]] == [256, 2, 16, 1] and C4.shape == (4, 5, 4)
    Y = mpg.to_mp(A, 128)
    name, a = rec.calls[-1]
    assert name == "mpgemm_terms_to_mp" and Y.shape == (6, 5, 3)
    assert [_v(x) for x in a[:5]] == [2, 15, A.data_ptr(), 128, Y.data_ptr()]
    X = mpg.from_mp(Y, 128, 4)
    name, a = rec.calls[-1]
    assert name == "mpgemm_mp_to_terms" and X.shape == (4, 5, 3)
    assert [_v(x) for x in a[:5]] == [4, 15, 128, Y.data_ptr(), X.data_ptr()]


def test_split_precision(rec):
    A, B = T(2, 5, 3), T(2, 3, 4)
    C = mpg.gemm_split(A, B, slices=12, digits="int8")
    name, a = rec.calls[-1]
    assert name == "mpgemm_dd_ozaki_ex"
    assert [_v(x) for x in a[:8]] == [5, 3, 4, A.data_ptr(), B.data_ptr(), C.data_ptr(), 12, 0]
    mpg.gemm_split(A, B)
    assert rec.calls[-1][0] == "mpgemm_dd_ozaki_ex" and [_v(x) for x in rec.calls[-1][1][6:8]] == [0, 1]
    A4, B4 = T(4, 5, 3), T(4, 3, 4)
    C4 = mpg.gemm_split(A4, B4, slices=40)
    name, a = rec.calls[-1]
    assert name == "mpgemm_qd_ozaki" and [_v(x) for x in a[:7]] == [5, 3, 4, A4.data_ptr(), B4.data_ptr(),
                                                                     C4.data_ptr(), 40]


def test_tuner_and_batched(rec):
    class Stream:
        cuda_stream = 77
    A, B, C = T(10, 5, 3, i32), T(10, 3, 4, i32), T(10, 5, 4, i32)
    tuner.tune("mp", A, B, C, flags=tuner.QUICK, prec_bits=256, stream=Stream())
    name, a = rec.calls[-1]
    assert name == "mpgemm_tune"
    assert [_v(x) for x in a[:10]] == [2, 256, 5, 3, 4, A.data_ptr(), B.data_ptr(), C.data_ptr(), tuner.QUICK, 77]
    D = [("dd", T(2, 5, 3), T(2, 3, 4), T(2, 5, 4)), ("qd", T(4, 2, 7), T(4, 7, 1), T(4, 2, 1)),
         ("mp256", T(10, 1, 1, i32), T(10, 1, 6, i32), T(10, 1, 6, i32))]
    descs = batched.make_descs(D, tiles=[16, 32, 16], integer_pipe=True)
    want = [(0, 0, 5, 3, 4, 16, 1), (1, 0, 2, 7, 1, 32, 1), (2, 256, 1, 1, 6, 16, 0)]
    for d, (fmt, A_, B_, C_), w in zip(descs, D, want):
        assert (d.kind, d.prec_bits, d.m, d.l, d.n, d.tile, d.engine) == w
        assert (d.A, d.B, d.C) == (A_.data_ptr(), B_.data_ptr(), C_.data_ptr())
