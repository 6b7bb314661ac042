"""The Python binding refuses malformed tensors before anything reaches the
library (no GPU).

Every public entry point checks its tensors' structure (planes, rows and
columns against the other operands, dtype, contiguity) and then that they
live on the GPU.  Host tensors of the right structure therefore reach the
last check and are refused as host tensors: the library is never handed a
host pointer, and there is no CPU path."""

import pytest

torch = pytest.importorskip("torch")
mpg = pytest.importorskip("paper_1710_01839_gb300")
from paper_1710_01839_gb300 import batched, tuner  # noqa: E402

f64, i32 = torch.float64, torch.int32


def T(planes, r, c, dtype=f64):
    return torch.zeros((planes, r, c), dtype=dtype)


def _host(fn):
    with pytest.raises(TypeError, match="CUDA tensor"):
        fn()


def test_well_formed_host_tensors_are_refused_as_host_tensors():
    _host(lambda: mpg.gemm_dd(T(2, 5, 3), T(2, 3, 4)))
    _host(lambda: mpg.gemm_dd(T(2, 5, 3), T(2, 3, 4), T(2, 5, 4)))
    _host(lambda: mpg.gemm_qd(T(4, 5, 3), T(4, 3, 4)))
    _host(lambda: mpg.gemm_mp(T(6, 5, 3, i32), T(6, 3, 4, i32), 128))
    _host(lambda: mpg.gemm_via_mp(T(2, 5, 3), T(2, 3, 4)))
    _host(lambda: mpg.gemm_via_mp(T(4, 5, 3), T(4, 3, 4), 256))
    _host(lambda: mpg.gemm_split(T(2, 5, 3), T(2, 3, 4)))
    _host(lambda: mpg.gemm_split(T(4, 5, 3), T(4, 3, 4)))
    _host(lambda: mpg.to_mp(T(2, 5, 3), 128))
    _host(lambda: mpg.from_mp(T(6, 5, 3, i32), 128, 2))
    _host(lambda: mpg.exponent_spread(T(2, 5, 3), T(2, 3, 4)))
    _host(lambda: tuner.tune("dd", T(2, 5, 3), T(2, 3, 4), T(2, 5, 4)))
    _host(lambda: tuner.tune("qd", T(4, 5, 3), T(4, 3, 4), T(4, 5, 4)))
    _host(lambda: tuner.tune("mp", T(10, 5, 3, i32), T(10, 3, 4, i32), T(10, 5, 4, i32), prec_bits=256))
    for fmt, planes, dt in (("dd", 2, f64), ("qd", 4, f64), ("mp256", 10, i32)):
        _host(lambda: batched.make_descs([(fmt, T(planes, 5, 3, dt), T(planes, 3, 4, dt), T(planes, 5, 4, dt))]))


@pytest.mark.parametrize("call", [
    lambda: mpg.gemm_dd(T(2, 5, 3), T(2, 4, 4)),                     # inner dimensions differ
    lambda: mpg.gemm_dd(T(2, 5, 3), T(2, 3, 4), T(2, 5, 5)),         # C's columns
    lambda: mpg.gemm_dd(T(2, 5, 3), T(2, 3, 4), T(2, 4, 4)),         # C's rows
    lambda: mpg.gemm_dd(T(3, 5, 3), T(3, 3, 4)),                     # planes
    lambda: mpg.gemm_dd(torch.zeros((2, 15), dtype=f64), T(2, 3, 4)),   # not (planes, rows, cols)
    lambda: mpg.gemm_dd(T(2, 3, 5).transpose(1, 2), T(2, 3, 4)),     # not contiguous
    lambda: mpg.gemm_qd(T(2, 5, 3), T(2, 3, 4)),                     # DD planes for QD
    lambda: mpg.gemm_mp(T(6, 5, 3, i32), T(6, 3, 4, i32), 256),      # planes of 128 bits for 256
    lambda: mpg.gemm_mp(T(6, 5, 3, i32), T(6, 3, 4, i32), 128, T(6, 5, 3, i32)),
    lambda: mpg.gemm_via_mp(T(3, 5, 3), T(3, 3, 4)),
    lambda: mpg.gemm_via_mp(T(2, 5, 3), T(2, 2, 4)),
    lambda: mpg.gemm_split(T(2, 5, 3), T(2, 3, 4), T(2, 5, 3)),
    lambda: mpg.gemm_split(T(4, 5, 3), T(4, 4, 4)),
    lambda: mpg.to_mp(T(3, 5, 3), 128),
    lambda: mpg.to_mp(T(2, 5, 3), 128, T(6, 5, 2, i32)),            # Y's columns
    lambda: mpg.to_mp(T(2, 5, 3), 128, T(10, 5, 3, i32)),           # Y's planes
    lambda: mpg.from_mp(T(6, 5, 3, i32), 128, 3),                   # 2 or 4 terms
    lambda: mpg.from_mp(T(6, 5, 3, i32), 128, 2, T(2, 4, 3)),       # X's rows
    lambda: mpg.exponent_spread(T(2, 5, 3), T(2, 4, 4)),
    lambda: tuner.tune("dd", T(2, 5, 3), T(2, 3, 4), T(2, 5, 5)),
    lambda: tuner.tune("mp", T(10, 5, 3, i32), T(10, 3, 4, i32), T(10, 5, 4, i32)),   # no prec_bits
    lambda: tuner.tune("mp", T(6, 5, 3, i32), T(6, 3, 4, i32), T(6, 5, 4, i32), prec_bits=256),
    lambda: batched.make_descs([("mp256", T(6, 4, 4, i32), T(6, 4, 4, i32), T(6, 4, 4, i32))]),
    lambda: batched.make_descs([("dd", T(2, 5, 3), T(2, 3, 4), T(2, 5, 5))]),
    lambda: batched.make_descs([("qd", T(4, 5, 3), T(4, 2, 4), T(4, 5, 4))]),
])
def test_malformed_tensors_are_refused(call):
    with pytest.raises(ValueError):
        call()


def test_wrong_dtypes_are_refused():
    with pytest.raises(TypeError, match="dtype"):
        mpg.gemm_dd(T(2, 5, 3, torch.float32), T(2, 3, 4))
    with pytest.raises(TypeError, match="dtype"):
        mpg.gemm_mp(T(6, 5, 3), T(6, 3, 4), 128)
    with pytest.raises(TypeError, match="torch tensor"):
        mpg.gemm_dd([[0.0]], T(2, 3, 4))
    with pytest.raises(TypeError, match="dtype"):
        batched.make_descs([("mp256", T(10, 4, 4), T(10, 4, 4), T(10, 4, 4))])


def test_cost_model_feature_rows_are_checked():
    import numpy as np
    from paper_1710_01839_gb300 import build, costmodel as cm
    build.build()                        # num_features() asks the (host-only) library
    nf = cm.num_features()
    for call in (lambda: cm.train(np.zeros((4, nf - 1)), np.ones(4)),      # columns
                 lambda: cm.train(np.zeros((4, nf)), np.ones(5)),          # rows against the times
                 lambda: cm.train(np.zeros((4, nf)), np.ones(4), epochs=0),
                 lambda: cm.predict(np.zeros((2, nf + 1))),
                 lambda: cm.predict(np.zeros(nf - 2))):
        with pytest.raises(ValueError):
            call()


def test_device_check_accepts_one_device_and_refuses_two():
    from paper_1710_01839_gb300._lib import require_cuda

    class OnDevice:                      # stands in for a CUDA tensor (is_cuda, device)
        def __init__(self, d):
            self.is_cuda, self.device = True, torch.device(d)

    require_cuda(A=OnDevice("cuda:0"), B=OnDevice("cuda:0"), C=OnDevice("cuda:0"))
    with pytest.raises(ValueError, match="cuda:1"):
        require_cuda(A=OnDevice("cuda:0"), B=OnDevice("cuda:1"))
    with pytest.raises(TypeError, match="CUDA tensor"):
        require_cuda(A=OnDevice("cuda:0"), B=torch.zeros(1))
