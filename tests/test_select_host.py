"""Precision selection from an accuracy target, host logic (no GPU, no cost
model loaded: measured static rates rank the candidates).

The a-priori bounds reproduce the library's defaults from first principles:
at a 2^-100 target with entries within one binade of their row / column
maxima, FP8 digits need S = 22 and int8 digits S = 16; DD's bound is
4 l 2^-104, QD's 4 l 2^-208, p-bit multi-limb gamma_l = l 2^-p / (1 - l 2^-p);
DD / QD on the integer pipe gamma_l(p) + 2^(1-p) + 2^(-53 T)."""

import math

import pytest

mpg = pytest.importorskip("paper_1710_01839_gb300")


@pytest.fixture(scope="module")
def built():
    try:
        mpg.lib()
    except Exception as e:   # library not built in this checkout
        pytest.skip(str(e))
    return mpg


def test_closed_form_bounds(built):
    assert built.precision_log2_bound("dd", 1024) == pytest.approx(2 + 10 - 104)
    assert built.precision_log2_bound("qd", 4096) == pytest.approx(2 + 12 - 208)
    lu = math.log2(1000) - 128
    assert built.precision_log2_bound("mp", 1000, prec_bits=128) == pytest.approx(lu - math.log2(1 - 2.0**lu))
    assert math.isnan(built.precision_log2_bound("ozaki_e4m3", 10, num_slices=25))
    assert math.isnan(built.precision_log2_bound("ozaki_int8", 10, num_slices=19))


@pytest.mark.parametrize("method,bits", [("ozaki_e4m3", 5), ("ozaki_int8", 7)])
def test_split_bounds_fall_with_slices_and_rise_with_spread(built, method, bits):
    prev = None
    for S in range(4, 19):
        b = built.precision_log2_bound(method, 4096, num_slices=S)
        if prev is not None and b > -100:
            assert prev - b == pytest.approx(bits, abs=0.5)   # one more digit: about b more bits
        assert b >= -106 - 1e-9                                  # the final DD rounding stays
        prev = b
    assert built.precision_log2_bound(method, 4096, num_slices=12, spread=5) > \
        built.precision_log2_bound(method, 4096, num_slices=12, spread=0) + 9


def test_integer_pipe_bounds(built):
    def via(l, p, T):
        lu = math.log2(l) - p
        g = 2.0 ** (lu - math.log2(1 - 2.0 ** lu))
        return math.log2((g + 2.0 ** (1 - p) + 2.0 ** (-53 * T)) * (1 + 2.0 ** -40))
    for l in (16, 1024, 1 << 20):
        assert built.precision_log2_bound("dd_via_mp", l) == pytest.approx(via(l, 128, 2), abs=1e-9)
        assert built.precision_log2_bound("qd_via_mp", l) == pytest.approx(via(l, 256, 4), abs=1e-9)
        assert built.precision_log2_bound("dd_via_mp", l, prec_bits=256) == pytest.approx(via(l, 256, 2), abs=1e-9)
    # the final expansion dominates: about 2^-106 (DD) and 2^-212 (QD), for any l
    assert -106.01 < built.precision_log2_bound("dd_via_mp", 4096) < -105.9
    assert -212.1 < built.precision_log2_bound("qd_via_mp", 4096) < -211.5
    assert math.isnan(built.precision_log2_bound("dd_via_mp", 64, prec_bits=96 + 1))
    # a DD target the FP64 kernels miss (4 l 2^-104 = 2^-92 at l = 1024) is met on the integer pipe
    sel = {c["method"]: c for c in built.select_precision(-104, 1024, 1024, 1024)}
    assert "dd" not in sel and sel["dd_via_mp"]["prec_bits"] == 128
    sel = {c["method"]: c for c in built.select_precision(-205, 1024, 1024, 1024)}
    assert "qd" not in sel and sel["qd_via_mp"]["prec_bits"] == 256


def test_defaults_reproduced(built):
    sel = {c["method"]: c for c in built.select_precision(-100, 4096, 4096, 4096)}
    assert sel["ozaki_e4m3"]["num_slices"] == 22
    assert sel["ozaki_int8"]["num_slices"] == 16
    assert "dd" not in sel                        # 4 * 4096 * 2^-104 = 2^-90
    assert sel["mp"]["prec_bits"] == 128
    assert "qd" in sel


def test_ranking_and_minimality(built):
    c = built.select_precision(-100, 4096, 4096, 4096)
    assert [x["method"] for x in c][:2] == ["ozaki_e4m3", "ozaki_int8"]
    assert all(c[i]["est_ms"] <= c[i + 1]["est_ms"] for i in range(len(c) - 1))
    for x in c:
        assert x["log2_bound"] <= -100
        if x["method"].startswith("ozaki"):       # one slice fewer would miss the target
            assert built.precision_log2_bound(x["method"], 4096, num_slices=x["num_slices"] - 1) > -100
    # a loose target lets DD in; a tight one leaves only the wide formats
    assert "dd" in {x["method"] for x in built.select_precision(-80, 1024, 1024, 1024)}
    qd = {x["method"]: x for x in built.select_precision(-200, 1024, 1024, 1024)}
    assert qd["ozaki_qd"]["num_slices"] == 42 and list(qd)[0] == "ozaki_qd"   # the QD split is fastest
    assert "ozaki_e4m3" not in qd and "dd" not in qd
    assert built.precision_log2_bound("ozaki_qd", 1024, num_slices=48) >= -211 - 1e-9
    tight = built.select_precision(-400, 256, 256, 256)
    assert [(x["method"], x["prec_bits"]) for x in tight] == [("mp", 512)]
    assert built.select_precision(-2000, 64, 64, 64) == []


def test_arguments(built):
    L = built.lib()
    assert L.mpgemm_select_precision(-100.0, 0, 1, 1, 0, None, 0) == -1
    assert L.mpgemm_select_precision(-100.0, 1, 1, 1, -1, None, 0) == -1
    assert L.mpgemm_select_precision(-100.0, 4, 4, 4, 0, None, 0) >= 1   # count only
