"""The tcgen05 level kernel's job order (mpgemm_split_job_order, the same
function the kernel evaluates per job), checked on the host before any
launch: every (tile, level) job appears exactly once, tiles start on the
128 x 256 grid inside C, levels run from S + 1 down to 2 within a
super-tile, and a super-tile's digit planes fit the L2 budget whenever a
super-tile is larger than one tile."""

import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def L():
    from paper_1710_01839_gb300 import build
    build.build()
    import paper_1710_01839_gb300 as mpg
    return mpg.lib()


def _order(L, m, n, l, S):
    J = L.mpgemm_split_job_order(m, n, l, S, None, 0)
    assert J > 0
    buf = (ctypes.c_int * (3 * J))()
    assert L.mpgemm_split_job_order(m, n, l, S, buf, J) == J
    return np.frombuffer(buf, dtype=np.int32).reshape(J, 3)


@pytest.mark.parametrize("m,n,l,S", [(4096, 4096, 4096, 22), (4096, 4096, 4096, 16), (1024, 1024, 1024, 44),
                                     (3000, 5000, 700, 24), (129, 257, 65536, 3), (37, 45, 70, 6),
                                     (8192, 2048, 8192, 22), (65535, 300, 512, 8), (520, 530, 300, 22)])
def test_every_job_once_in_super_tile_order(L, m, n, l, S):
    jobs = _order(L, m, n, l, S)
    tm, tn = -(-m // 128), -(-n // 256)
    assert len(jobs) == tm * tn * S
    g, r0, c0 = jobs[:, 0], jobs[:, 1], jobs[:, 2]
    assert ((r0 % 128) == 0).all() and ((c0 % 256) == 0).all()
    assert (r0 >= 0).all() and (r0 < m).all() and (c0 >= 0).all() and (c0 < n).all()
    assert ((g >= 2) & (g <= S + 1)).all()
    keys = set(zip(g.tolist(), (r0 // 128).tolist(), (c0 // 256).tolist()))
    assert len(keys) == len(jobs)                      # a bijection onto tiles x levels
    # super-tiles: maximal runs of jobs over one set of tiles, levels descending
    lp = -(-l // 128) * 128
    i = 0
    while i < len(jobs):
        tiles = set()
        j = i
        while j < len(jobs) and g[j] == S + 1:
            tiles.add((r0[j], c0[j]))
            j += 1
        k = j + (len(tiles) * (S - 1))
        block = jobs[i:k]
        assert len(block) == len(tiles) * S
        for lvl in range(S):
            part = block[lvl * len(tiles):(lvl + 1) * len(tiles)]
            assert (part[:, 0] == S + 1 - lvl).all()
            assert set(zip(part[:, 1], part[:, 2])) == tiles
        rows = {r for r, _ in tiles}
        cols = {c for _, c in tiles}
        assert len(tiles) == len(rows) * len(cols)      # a rectangle of tiles
        if len(tiles) > 1:
            assert (len(rows) * 128 + len(cols) * 256) * lp * S <= 96 * 2**20
        i = k


def test_small_problems_keep_the_level_major_order(L):
    jobs = _order(L, 1024, 1024, 1024, 44)
    # everything fits one super-tile: all tiles of level S + 1, then level S, ...
    assert (np.diff(jobs[:, 0]) <= 0).all()


def test_arguments(L):
    assert L.mpgemm_split_job_order(0, 4, 4, 2, None, 0) == -1
    assert L.mpgemm_split_job_order(4, 70000, 4, 2, None, 0) == -1
    assert L.mpgemm_split_job_order(4, 4, 4, 2, None, 5) == -1
