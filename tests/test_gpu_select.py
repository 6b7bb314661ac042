"""Precision selection on the GPU: the exponent spread computed by the
library equals its definition on the hi words, and the configurations the
selector returns for a target meet it on real products (measured against
the exact product on sampled entries)."""

import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import dev, host, sample_indices
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")


def _spread_def(A, B):
    """max over rows of A / columns of B of (largest - smallest nonzero frexp exponent) of the hi words."""
    def rows(X):
        e = np.frexp(X)[1].astype(np.int64)
        nz = X != 0
        hi = np.where(nz, e, -10**9).max(axis=1)
        lo = np.where(nz, e, 10**9).min(axis=1)
        return int(np.max(np.where(nz.any(axis=1), hi - lo, 0)))
    return max(rows(A[0]), rows(B[0].T))


def test_exponent_spread_matches_definition():
    A, B = I.dd_rowcol_scaled(70, 300, 90, seed=3)
    A[:, 4, :] = 0.0
    B[:, :, 5] = 0.0
    A[0, 7, 3] = 2.0**-900          # one tiny entry widens row 7
    A[1, 7, 3] = 0.0
    assert mpg.exponent_spread(dev(A), dev(B)) == _spread_def(A, B)
    Z = np.zeros((2, 8, 8))
    assert mpg.exponent_spread(dev(Z), dev(Z)) == 0


@pytest.mark.parametrize("target", [-60, -90, -100])
def test_selected_configurations_meet_target(target):
    import torch
    m, l, n = 384, 512, 320
    A, B = I.dd_rowcol_scaled(m, l, n, seed=I.seed_for(3, -target))
    Ad, Bd = dev(A), dev(B)
    spread = mpg.exponent_spread(Ad, Bd)
    choices = mpg.select_precision(target, m, l, n, spread=spread)
    assert choices, "no configuration meets the target"
    ii, jj = sample_indices(m, n, 300, seed=-target)
    sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for c in choices:
        if c["method"] not in ("ozaki_e4m3", "ozaki_int8", "dd", "dd_via_mp"):
            continue
        if c["method"] == "dd":
            C = host(mpg.gemm_dd(Ad, Bd, algo="block"))
        elif c["method"] == "dd_via_mp":
            C = host(mpg.gemm_via_mp(Ad, Bd, c["prec_bits"], algo="block", n_min=16))
        else:
            Cd = torch.empty((2, m, n), dtype=torch.float64, device="cuda")
            kind = 1 if c["method"] == "ozaki_e4m3" else 0
            assert mpg.lib().mpgemm_dd_ozaki_ex(m, l, n, ctypes.c_void_p(Ad.data_ptr()),
                                                ctypes.c_void_p(Bd.data_ptr()), ctypes.c_void_p(Cd.data_ptr()),
                                                c["num_slices"], kind, sp) == 0
            C = host(Cd)
        err, absab = oracle.exact_check(A, B, C, ii, jj)
        assert np.max(err / absab) <= 2.0**c["log2_bound"] <= 2.0**target, c
