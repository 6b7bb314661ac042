"""Out-of-bounds accesses, checked without a sanitizer: every operand,
output and the library workspace is placed between guard zones (NaN for
doubles, a fixed bit pattern for multi-limb words), and every GEMM path runs
at ragged sizes (not multiples of any tile, Strassen's zero extension at
work).  A write past a buffer changes a guard zone; a read past an operand
brings NaN or the pattern into the result, which then differs from the same
call on plain buffers.  Both are checked for DD / QD (simple, block, every
tile, Strassen depths 1-4), multi-limb (128 / 256 / 1024 bits), split
precision (int8 and FP8 digits, DD and QD), DD / QD on the integer pipe and
a batched plan."""

import ctypes

import numpy as np
import pytest

from gpu_util import host
from paper_1710_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

mpg = pytest.importorskip("paper_1710_01839_gb300")

GUARD_BYTES = 4096           # keeps every view 4 KB aligned, like a fresh allocation
PATTERN = 0x7FC5A5A5         # multi-limb guard word (never written by the kernels as a whole zone)


class Guarded:
    """A tensor of `shape` inside a buffer with guard zones on both sides."""

    def __init__(self, shape, dtype, fill=None):
        import torch
        self.dtype = dtype
        es = torch.empty((), dtype=dtype).element_size()
        self.g = GUARD_BYTES // es
        n = int(np.prod(shape))
        if dtype == torch.float64:
            self.full = torch.full((self.g + n + self.g,), float("nan"), dtype=dtype, device="cuda")
        else:
            self.full = torch.full((self.g + n + self.g,), PATTERN, dtype=dtype, device="cuda")
        self.t = self.full[self.g:self.g + n].view(*shape)
        if fill is not None:
            self.t.copy_(fill)
        self.before = self.full[:self.g].clone()
        self.after = self.full[self.g + n:].clone()

    def intact(self):
        import torch
        b, a = self.full[:self.g], self.full[-self.g:]
        if self.dtype == torch.float64:
            same = lambda x, y: bool(torch.equal(x.view(torch.int64), y.view(torch.int64)))
        else:
            same = lambda x, y: bool(torch.equal(x, y))
        return same(b, self.before) and same(a, self.after)


def _dd_like(planes, rows, cols, seed):
    gen = I.dd_random if planes == 2 else I.qd_random
    return gen(rows, cols, seed, exp_spread=20)


def _workspace(nbytes):
    import torch
    ws = Guarded((nbytes // 8 + 1,), torch.float64)
    ws.t.zero_()
    ws.before, ws.after = ws.full[:ws.g].clone(), ws.full[-ws.g:].clone()
    rc = mpg.lib().mpgemm_set_workspace(ctypes.c_void_p(ws.t.data_ptr()), ws.t.numel() * 8)
    assert rc == 0
    return ws


@pytest.fixture(autouse=True)
def _no_workspace_after():
    yield
    mpg.lib().mpgemm_set_workspace(None, 0)


@pytest.mark.parametrize("fmt", ["dd", "qd"])
@pytest.mark.parametrize("m,l,n", [(37, 53, 71), (130, 255, 97), (257, 129, 300)])
def test_dd_qd_all_algorithms(fmt, m, l, n):
    import torch
    P = 2 if fmt == "dd" else 4
    f = mpg.gemm_dd if fmt == "dd" else mpg.gemm_qd
    A, B = _dd_like(P, m, l, 5), _dd_like(P, l, n, 6)
    Ag, Bg = Guarded((P, m, l), torch.float64, torch.from_numpy(A)), Guarded((P, l, n), torch.float64, torch.from_numpy(B))
    Ap, Bp = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    ws = _workspace(max(mpg.workspace_size(fmt, m, l, n, algo="strassen", depth=d) for d in (1, 2, 3, 4)))
    tiles = (16, 32, 64) if fmt == "dd" else (16, 32)
    configs = [("simple", 16, 0)] + [("block", t, 0) for t in tiles] + [("strassen", t, d) for t in tiles[:2]
                                                                         for d in (1, 2, 3, 4)]
    for algo, nm, d in configs:
        Cg = Guarded((P, m, n), torch.float64)
        f(Ag.t, Bg.t, Cg.t, algo=algo, n_min=nm, depth=d)
        want = host(f(Ap, Bp, algo=algo, n_min=nm, depth=d))
        got = host(Cg.t)
        assert np.isfinite(got).all(), (algo, nm, d)
        assert np.array_equal(got, want), (algo, nm, d)
        assert Cg.intact() and Ag.intact() and Bg.intact() and ws.intact(), (algo, nm, d)
    assert mpg.stream_status() == 0


@pytest.mark.parametrize("bits", [128, 256, 1024])
def test_multi_limb_all_algorithms(bits):
    import torch
    m, l, n = 45, 67, 39
    w = bits // 32
    A = I.mp_random(m, l, w, 7).view(np.int32)
    B = I.mp_random(l, n, w, 8).view(np.int32)
    Ag = Guarded((2 + w, m, l), torch.int32, torch.from_numpy(A))
    Bg = Guarded((2 + w, l, n), torch.int32, torch.from_numpy(B))
    Ap, Bp = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    ws = _workspace(max(mpg.workspace_size("mp", m, l, n, algo="strassen", depth=d, prec_bits=bits) for d in (1, 2, 3)))
    for algo, nm, d in [("simple", 16, 0), ("block", 16, 0), ("block", 64, 0), ("strassen", 16, 1),
                        ("strassen", 16, 2), ("strassen", 16, 3)]:
        Cg = Guarded((2 + w, m, n), torch.int32)
        mpg.gemm_mp(Ag.t, Bg.t, bits, Cg.t, algo=algo, n_min=nm, depth=d)
        want = host(mpg.gemm_mp(Ap, Bp, bits, algo=algo, n_min=nm, depth=d), mp=True)
        assert np.array_equal(host(Cg.t, mp=True), want), (algo, d)
        assert Cg.intact() and Ag.intact() and Bg.intact() and ws.intact(), (algo, d)
    assert mpg.stream_status() == 0


@pytest.mark.parametrize("fmt,digits,S", [("dd", "int8", 16), ("dd", "e4m3", 22), ("qd", "e4m3", 44)])
def test_split_precision(fmt, digits, S):
    import torch
    m, l, n = 131, 300, 261
    P = 2 if fmt == "dd" else 4
    if fmt == "dd":
        A, B = I.dd_rowcol_scaled(m, l, n, seed=9)
    else:
        A, B = I.qd_rowcol_scaled(m, l, n, seed=9)
    Ag, Bg = Guarded((P, m, l), torch.float64, torch.from_numpy(A)), Guarded((P, l, n), torch.float64, torch.from_numpy(B))
    Ap, Bp = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    ws = _workspace(int(mpg.lib().mpgemm_ozaki_workspace_size(m, l, n, S)))
    Cg = Guarded((P, m, n), torch.float64)
    mpg.gemm_split(Ag.t, Bg.t, Cg.t, slices=S, digits=digits)
    want = host(mpg.gemm_split(Ap, Bp, slices=S, digits=digits))
    assert np.array_equal(host(Cg.t), want)
    assert Cg.intact() and Ag.intact() and Bg.intact() and ws.intact()
    assert mpg.stream_status() == 0


@pytest.mark.parametrize("fmt,bits", [("dd", 128), ("qd", 256)])
def test_integer_pipe(fmt, bits):
    import torch
    m, l, n = 77, 150, 91
    P = 2 if fmt == "dd" else 4
    A, B = _dd_like(P, m, l, 11), _dd_like(P, l, n, 12)
    Ag, Bg = Guarded((P, m, l), torch.float64, torch.from_numpy(A)), Guarded((P, l, n), torch.float64, torch.from_numpy(B))
    Ap, Bp = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    ws = _workspace(64 << 20)
    for algo, d in [("block", 0), ("strassen", 2)]:
        Cg = Guarded((P, m, n), torch.float64)
        mpg.gemm_via_mp(Ag.t, Bg.t, bits, Cg.t, algo=algo, n_min=16, depth=d)
        want = host(mpg.gemm_via_mp(Ap, Bp, bits, algo=algo, n_min=16, depth=d))
        assert np.array_equal(host(Cg.t), want), algo
        assert Cg.intact() and Ag.intact() and Bg.intact() and ws.intact(), algo
    assert mpg.stream_status() == 0


def test_batched_plan():
    import torch
    from paper_1710_01839_gb300 import batched
    shapes = [("dd", 33, 47, 65), ("qd", 70, 19, 40), ("mp256", 21, 90, 17), ("dd", 129, 31, 140)]
    guarded, plain = [], []
    for i, (fmt, m, l, n) in enumerate(shapes):
        if fmt == "mp256":
            A = I.mp_random(m, l, 8, 30 + i).view(np.int32)
            B = I.mp_random(l, n, 8, 40 + i).view(np.int32)
            P, dt = 10, torch.int32
        else:
            P = 2 if fmt == "dd" else 4
            A, B, dt = _dd_like(P, m, l, 30 + i), _dd_like(P, l, n, 40 + i), torch.float64
        g = (fmt, Guarded((P, m, l), dt, torch.from_numpy(A)), Guarded((P, l, n), dt, torch.from_numpy(B)),
             Guarded((P, m, n), dt))
        guarded.append(g)
        plain.append((fmt, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                      torch.zeros((P, m, n), dtype=dt, device="cuda")))
    for integer_pipe in (False, True):
        dg = batched.make_descs([(f, a.t, b.t, c.t) for f, a, b, c in guarded], integer_pipe=integer_pipe)
        dp = batched.make_descs(plain, integer_pipe=integer_pipe)
        plan = batched.Plan(dg)
        plan.run_graph()
        plan.close()
        batched.sequential(dp)
        for (fmt, a, b, c), (_, _, _, cp) in zip(guarded, plain):
            mp = fmt == "mp256"
            assert np.array_equal(host(c.t, mp=mp), host(cp, mp=mp)), (fmt, integer_pipe)
            assert a.intact() and b.intact() and c.intact(), (fmt, integer_pipe)
    assert mpg.stream_status() == 0
