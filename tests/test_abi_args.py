"""Argument checks of the C ABI that return before any CUDA call (no GPU).

Every case here must be refused by the entry point's own checks (sizes,
algorithm, n_min, depth, NULL and overlapping buffers, precision, slice
counts, documented size limits), so the placeholder addresses passed for A,
B and C are never touched.  The test is skipped wherever a CUDA device is
visible, so that a check that failed to refuse could never launch work on
those addresses."""

import ctypes

import pytest

EINVAL, EUNSUPPORTED = -1, -2
SIMPLE, BLOCK, STRASSEN, AUTO = 0, 1, 2, 3

# far apart, never dereferenced
PA, PB, PC = ctypes.c_void_p(1 << 40), ctypes.c_void_p(2 << 40), ctypes.c_void_p(3 << 40)
NULL = None


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("placeholder-pointer checks run only where no GPU is visible")
    from paper_1710_01839_gb300 import build
    build.build()
    import paper_1710_01839_gb300 as mpg
    return mpg.lib()


DDQD_CASES = [
    # (m, l, n, A, B, C, algo, n_min, depth) -> code
    ((-1, 4, 4, PA, PB, PC, BLOCK, 0, 0), EINVAL),
    ((4, -1, 4, PA, PB, PC, BLOCK, 0, 0), EINVAL),
    ((4, 4, -1, PA, PB, PC, BLOCK, 0, 0), EINVAL),
    (((1 << 31) + 1, 4, 4, PA, PB, PC, BLOCK, 0, 0), EINVAL),
    ((4, 4, 4, PA, PB, PC, 4, 0, 0), EINVAL),               # no such algorithm
    ((4, 4, 4, PA, PB, PC, -1, 0, 0), EINVAL),
    ((4, 4, 4, PA, PB, PC, BLOCK, 48, 0), EINVAL),          # n_min not a power of two
    ((4, 4, 4, PA, PB, PC, BLOCK, 2048, 0), EINVAL),        # n_min above 1024
    ((4, 4, 4, PA, PB, PC, STRASSEN, 0, 5), EINVAL),        # depth above 4
    ((4, 4, 4, PA, PB, PC, STRASSEN, 0, -1), EINVAL),
    ((4, 4, 4, NULL, PB, PC, BLOCK, 0, 0), EINVAL),
    ((4, 4, 4, PA, NULL, PC, BLOCK, 0, 0), EINVAL),
    ((4, 4, 4, PA, PB, NULL, BLOCK, 0, 0), EINVAL),
    ((4, 4, 4, PA, PB, PA, BLOCK, 0, 0), EINVAL),           # C is A
    ((4, 4, 4, PA, PB, ctypes.c_void_p((1 << 40) + 64), BLOCK, 0, 0), EINVAL),   # C overlaps A
    ((4, 4, 4, PA, PB, ctypes.c_void_p((2 << 40) - 64), BLOCK, 0, 0), EINVAL),   # C runs into B
    ((140000, 4, 4, PA, PB, PC, STRASSEN, 0, 1), EUNSUPPORTED),   # a half's rows beyond grid.y
]


@pytest.mark.parametrize("fn", ["mpgemm_dd", "mpgemm_qd"])
@pytest.mark.parametrize("args,code", DDQD_CASES)
def test_dd_qd_refuse_bad_arguments(L, fn, args, code):
    assert getattr(L, fn)(*args, None) == code


@pytest.mark.parametrize("args,code", DDQD_CASES)
def test_mp_refuses_bad_arguments(L, args, code):
    m, l, n, A, B, C, algo, n_min, depth = args
    assert L.mpgemm_mp(m, l, n, 256, A, B, C, algo, n_min, depth, None) == code


@pytest.mark.parametrize("prec,code", [(0, EINVAL), (-32, EINVAL), (48, EINVAL), (96, EUNSUPPORTED),
                                       (4096, EUNSUPPORTED)])
def test_mp_refuses_bad_precision(L, prec, code):
    assert L.mpgemm_mp(4, 4, 4, prec, PA, PB, PC, BLOCK, 0, 0, None) == code


@pytest.mark.parametrize("fn", ["mpgemm_dd_via_mp", "mpgemm_qd_via_mp"])
def test_via_mp_refuses_bad_arguments(L, fn):
    f = getattr(L, fn)
    # the integer-pipe width must be 64, 128, 256 or 512 bits
    for prec in (0, 32, 96, 1024):
        assert f(4, 4, 4, PA, PB, PC, prec, BLOCK, 0, 0, None) == EUNSUPPORTED
    for args, code in DDQD_CASES:
        m, l, n, A, B, C, algo, n_min, depth = args
        assert f(m, l, n, A, B, C, 128, algo, n_min, depth, None) == code


def test_terms_to_mp_refuses_bad_arguments(L):
    assert L.mpgemm_terms_to_mp(3, 16, PA, 128, PC, None) == EINVAL       # 2 or 4 terms only
    assert L.mpgemm_terms_to_mp(2, 16, PA, 96, PC, None) == EUNSUPPORTED


@pytest.mark.parametrize("args,code", [
    ((4, 4, 4, PA, PB, PC, 16, 2), EINVAL),                 # no such digit kind
    ((-1, 4, 4, PA, PB, PC, 16, 0), EINVAL),
    ((4, 4, 4, NULL, PB, PC, 16, 0), EINVAL),
    ((4, 4, 4, PA, PB, NULL, 16, 1), EINVAL),
    ((4, 4, 4, PA, PB, PC, 1000, 0), EINVAL),               # more slices than the pipeline takes (18 int8, 24 FP8)
    ((4, 4, 4, PA, PB, PC, 1000, 1), EINVAL),
    ((4, 10000, 4, PA, PB, PC, 16, 0), EUNSUPPORTED),       # int8: S 127^2 l reaches 2^31
    ((4, 70000, 4, PA, PB, PC, 22, 1), EUNSUPPORTED),       # FP8: a pair's f32 sum reaches 2^24
    ((70000, 4, 4, PA, PB, PC, 16, 0), EUNSUPPORTED),       # rows beyond grid.y of the slice kernels
])
def test_split_precision_refuses_bad_arguments(L, args, code):
    m, l, n, A, B, C, S, kind = args
    assert L.mpgemm_dd_ozaki_ex(m, l, n, A, B, C, S, kind, None) == code
