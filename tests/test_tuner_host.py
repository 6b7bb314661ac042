"""The predictor of Section 3 against the paper's own numbers (no GPU).

Tables 1 and 3 print, for n = 1024, the time of the sampled run (c) and the
predicted full time (d); in all 44 rows d = c * 1024 / r with r = 2 n_min
(r = n when 2 n_min >= n) up to the tables' 3-digit printing.  The library's
prediction (mpgemm_predict_time) with the library's sample-row rule
(mpgemm_sample_rows, here on a 1-SM machine so the wave floor is inactive)
must reproduce column (d) from column (c), and the printed rel.diff must be
|d - b| / b.
"""

import csv
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _rows():
    with open(os.path.join(HERE, "golden", "paper_tables_1_3.csv")) as f:
        lines = [ln for ln in f if not ln.startswith("#")]
    return list(csv.DictReader(lines))


@pytest.fixture(scope="module")
def tuner():
    from paper_1710_01839_gb300 import build
    build.build()
    from paper_1710_01839_gb300 import tuner as t
    return t


def test_fixture_complete():
    rows = _rows()
    assert len(rows) == 44
    assert sum(r["table"] == "1" for r in rows) == 22


def test_prediction_reproduces_tables(tuner):
    n = 1024
    for r in _rows():
        n_min = int(r["n_min"])
        fmt = "dd" if r["prec"] in ("DD", "QD") else "mp"
        rows = tuner.sample_rows("dd", n, n, n_min, num_sms=1) if fmt == "dd" else min(n, 2 * n_min)
        assert rows == min(n, 2 * n_min)
        pred = tuner.predict_time(float(r["c_sample_s"]), n, rows)
        d = float(r["d_pred_s"])
        # (c) and (d) are printed to 3 significant digits
        assert abs(pred - d) <= 0.012 * d, (r, pred)


def test_printed_rel_diff_is_relative_difference():
    for r in _rows():
        b, d, pct = float(r["b_block_s"]), float(r["d_pred_s"]), float(r["reldiff_pct"])
        assert abs(100 * abs(d - b) / b - pct) <= 0.02 * max(pct, 1.0) + 0.02, r


def test_paper_acceptance_threshold():
    # every printed prediction is within 10 % (the paper's bound) of the real time
    assert max(float(r["reldiff_pct"]) for r in _rows()) < 10.0


def test_sample_rows_rule(tuner):
    # at least 2 n_min, at least one wave of CTAs, a multiple of the CTA tile, at most m
    assert tuner.sample_rows("dd", 2048, 2048, 64, num_sms=1) == 128
    assert tuner.sample_rows("dd", 1024, 1024, 512, num_sms=1) == 1024
    r = tuner.sample_rows("dd", 2048, 2048, 16, num_sms=152)   # 16-tiles: 128 per row of tiles
    assert r % 16 == 0 and r >= 32 and (r // 16) * (2048 // 16) >= 152 * 4
    assert tuner.sample_rows("qd", 100, 100, 256, num_sms=152) == 100
    assert tuner.predict_time(2.0, 1024, 128) == 16.0
