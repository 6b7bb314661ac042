"""The FP32 MLP cost model on the GPU: the hand-written training kernel fits a
known function, fits measured timings, round-trips through a file, and
drives MPGEMM_AUTO to valid configurations."""

import numpy as np
import pytest

from gpu_util import DD_BOUND, dev, host, sample_indices
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")


def _random_configs(cm, count, seed):
    rng = np.random.default_rng(seed)
    F = []
    for _ in range(count):
        m, l, n = (int(x) for x in np.exp(rng.uniform(np.log(16), np.log(1024), 3)))
        kind = ["dd", "qd", "mp"][rng.integers(0, 3)]
        algo = ["simple", "block"][rng.integers(0, 2)]
        tile = [16, 32][rng.integers(0, 2)]
        F.append(cm.features(kind, m, l, n, algo, tile, prec_bits=256 if kind == "mp" else 0))
    return np.array(F)


def test_training_kernel_fits_a_known_function():
    from paper_1710_01839_gb300 import costmodel as cm
    F = _random_configs(cm, 2560, 1)
    # a smooth nonlinear "time": work x format cost, plus a wave-quantisation term
    t = np.exp(0.69 * (F[:, 3] - 27) + 2.0 * F[:, 5] + 1.2 * F[:, 6] + 0.4 * np.maximum(F[:, 14] - 2, 0) - 0.3 * F[:, 8])
    tr, te = slice(0, 2304), slice(2304, 2560)
    loss = cm.train(F[tr], t[tr], epochs=300, seed=3)
    assert loss[-1] < 0.05 * loss[0]
    pred = cm.predict(F[te])
    rel = np.abs(pred / t[te] - 1)
    assert np.median(rel) < 0.10, np.median(rel)
    cm.clear()


def test_real_timings_fit_roundtrip_and_auto(tmp_path):
    from paper_1710_01839_gb300 import costmodel as cm
    F, T = cm.collect(1024, seed=7, max_dim=384)
    assert np.all(T > 0) and np.all(np.isfinite(F))
    loss = cm.train(F[:896], T[:896], epochs=200, seed=1)
    assert loss[-1] < 0.5 * loss[0]
    pred = cm.predict(F[896:])
    rel = np.abs(pred / T[896:] - 1)
    assert np.median(rel) < 0.35, np.median(rel)
    path = str(tmp_path / "model.bin")
    cm.save(path)
    p1 = cm.predict(F[:50])
    cm.clear()
    with pytest.raises(mpg.MpgemmError):
        cm.predict(F[:1])
    cm.load(path)
    assert np.array_equal(p1, cm.predict(F[:50]))
    # AUTO without a remembered tuning uses the model; the result meets the DD bound
    mpg.lib().mpgemm_tune_forget()
    n = 256
    A, B = I.dd_random(n, n, 31), I.dd_random(n, n, 32)
    C = host(mpg.gemm_dd(dev(A), dev(B), algo="auto"))
    ii, jj = sample_indices(n, n, 128, seed=2)
    import oracle
    err, absab = oracle.exact_check(A, B, C, ii, jj)
    amax, bmax = np.max(np.abs(A[0])), np.max(np.abs(B[0]))
    # whichever algorithm the model picked: the DD bound (or the Strassen bound)
    assert np.all((err <= DD_BOUND * n * absab) | (err <= 2.0**-96 * n * amax * bmax))
    cm.clear()
