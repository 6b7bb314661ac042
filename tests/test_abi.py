"""The C-ABI library loads and exports every entry point the public header
declares (no GPU needed: nothing is launched).  Host-only calls that touch
no device (strerror, version, workspace sizing) are exercised too."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(mpgemm_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    from paper_1710_01839_gb300 import build
    build.build()
    import paper_1710_01839_gb300 as mpg
    return mpg


def test_header_declares_entry_points():
    names = _declared_functions()
    for want in ("mpgemm_dd", "mpgemm_qd", "mpgemm_mp", "mpgemm_stream_status", "mpgemm_workspace_size"):
        assert want in names


def test_library_exports_every_declared_symbol(built):
    L = built.lib()
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_declares_every_symbol(built):
    from paper_1710_01839_gb300 import _lib
    assert set(_declared_functions()) <= set(_lib.SIGNATURES)


def test_host_only_calls(built):
    L = built.lib()
    assert built.strerror(0) == "ok"
    assert "invalid" in built.strerror(-1)
    assert L.mpgemm_version() >= 100
    # workspace sizing is host arithmetic
    assert built.workspace_size("dd", 64, 64, 64, algo="block") == 0
    w1 = built.workspace_size("dd", 64, 64, 64, algo="strassen", depth=1)
    assert w1 >= 7 * 3 * 32 * 32 * 16
    assert built.workspace_size("dd", 64, 64, 64, algo="strassen", depth=2) > w1
    assert built.workspace_size("mp", 64, 64, 64, algo="strassen", depth=1, prec_bits=256) > 0
    # odd sizes are zero-extended: the workspace is that of the extended problem
    assert built.workspace_size("dd", 63, 63, 63, algo="strassen", depth=2) == \
        built.workspace_size("dd", 64, 64, 64, algo="strassen", depth=2)
    # argument checks that return before any CUDA call
    assert L.mpgemm_selftest_wait_timeout(0, None) == -1
    assert L.mpgemm_selftest_wait_timeout(5000, None) == -1
    assert L.mpgemm_stream_sms is not None
    import ctypes
    ops = ctypes.c_double()
    assert L.mpgemm_peak_run(7, 1, ctypes.byref(ops), None) == -1           # unknown kind
    assert L.mpgemm_peak_run(0, 0, ctypes.byref(ops), None) == -1           # no iterations
    assert L.mpgemm_peak_run(0, (1 << 22) + 1, ctypes.byref(ops), None) == -1   # tcgen05 loop too long
    assert L.mpgemm_peak_run(2, 1, None, None) == -1                        # no ops output
    # the multi-limb leaf setting is host state: returns the previous value
    assert L.mpgemm_set_mp_leaf(2) == 0
    assert L.mpgemm_set_mp_leaf(1) == 2
    assert L.mpgemm_set_mp_leaf(3) == -1 and L.mpgemm_set_mp_leaf(-1) == -1
    assert L.mpgemm_set_mp_leaf(0) == 1
    assert built.set_mp_leaf("team") == "default" and built.set_mp_leaf("default") == "team"
    import pytest
    with pytest.raises(ValueError):
        built.set_mp_leaf("warp")
    # which multi-limb block kernel a call uses (host arithmetic): the team
    # kernel at 512-2048 bits when the one-thread grid (16 x 16 per CTA)
    # has at most one CTA per two SMs
    choice = L.mpgemm_mp_leaf_choice
    assert choice(1024, 128, 128, 1, 152) == 2          # 64 CTAs <= 76
    assert choice(1024, 144, 128, 1, 152) == 2          # 72
    assert choice(1024, 160, 128, 1, 152) == 1          # 80 > 76
    assert choice(1024, 64, 64, 4, 152) == 2 and choice(1024, 64, 64, 7, 152) == 1   # 64 and 112 CTAs
    assert choice(1024, 128, 128, 1, 24) == 1           # a 24-SM partition: 64 > 12
    assert choice(256, 16, 16, 1, 152) == 1 and choice(4096, 16, 16, 1, 152) == 1   # other widths
    assert choice(512, 16, 16, 1, 152) == 2 and choice(2048, 1, 1, 1, 152) == 2
    assert choice(100, 16, 16, 1, 152) == -1 and choice(512, 16, 16, 0, 152) == -1 and choice(512, 1, 1, 1, 0) == -1
    assert L.mpgemm_set_mp_leaf(1) == 0
    assert choice(2048, 16, 16, 1, 152) == 1
    assert L.mpgemm_set_mp_leaf(2) == 1
    assert choice(2048, 4096, 4096, 1, 152) == 2
    assert L.mpgemm_set_mp_leaf(0) == 2
    # the bounds counter exists only in the bounds-checked build
    assert L.mpgemm_bounds_read(None, None) == -2 and L.mpgemm_selftest_bounds(None) == -2
    # the arithmetic self-tests check their arguments before any CUDA call:
    # a negative count or missing buffers are refused, an empty one is a no-op
    buf = ctypes.c_void_p(8)                 # never dereferenced: refused or count 0
    for name in ("mpgemm_selftest_two_sum", "mpgemm_selftest_two_prod"):
        f = getattr(L, name)
        assert f(-1, buf, buf, buf, None) == -1, name
        assert f(4, None, buf, buf, None) == -1 and f(4, buf, None, buf, None) == -1, name
        assert f(4, buf, buf, None, None) == -1, name
        assert f(0, None, None, None, None) == 0, name
    for name in ("mpgemm_selftest_dd_mac", "mpgemm_selftest_dd_add"):
        f = getattr(L, name)
        assert f(-1, buf, buf, None) == -1, name
        assert f(4, None, buf, None) == -1 and f(4, buf, None, None) == -1, name
        assert f(0, None, None, None) == 0, name


def test_checked_build_exists_and_exports(built):
    import ctypes
    from paper_1710_01839_gb300._lib import lib_checked, SIGNATURES
    Lc = lib_checked()
    for name in SIGNATURES:
        assert hasattr(Lc, name), name
    c, f = ctypes.c_longlong(), ctypes.c_ulonglong()
    assert Lc.mpgemm_bounds_read(None, ctypes.byref(f)) == -1        # argument check before any device call
    assert Lc.mpgemm_version() == built.lib().mpgemm_version()
