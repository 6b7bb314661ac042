"""MPGEMM_AUTO's picks against exhaustive timing: the shipped cost model
decides, and when more than one configuration is predicted within its own
error of the best it times that short list once on the operands (the
paper's Section 3 idea: predict to prune, time the finalists).  On a fixed
subset of 24 shapes drawn like the batched workload (m, l, n log-uniform in
[16, 1024]; DD, QD, 256- and 128-bit), every pick must be within 10 % of the
fastest configuration timed exhaustively.  Both sides use the library's
timer (calls issued back to back from C between two events, the
steady-state cost of a call; the exhaustive side takes medians of windows
interleaved over the candidates): at sizes of a few tens of microseconds a
timer in Python would measure its own per-call overhead instead.  A
difference below 3 microseconds, the size of launch jitter, counts as a
tie."""

import os

import pytest

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")


def test_auto_regret_within_ten_percent_on_fixed_shapes():
    from paper_1710_01839_gb300 import costmodel as cm, train_cost_model as tcm
    if not os.path.exists(cm.DEFAULT_MODEL):
        pytest.skip("no shipped cost model")
    cm.load(cm.DEFAULT_MODEL)
    try:
        res = tcm.auto_regret_study(tcm.batched_like_shapes(24, seed=2024), reps=7)
    finally:
        mpg.lib().mpgemm_tune_forget()
    bad = [r for r in res["shapes"]
           if r["regret_auto"] > 0.10 and (r["t_auto_ms"] - r["t_best_ms"]) * 1e3 > 3.0]
    assert not bad, bad
