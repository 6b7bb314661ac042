"""The persistent tuning cache on the GPU: one process runs the Section 3
procedure on device timings with a cache file open; a second process opens
the file, gets the same choice back without timing anything, and
MPGEMM_AUTO in that process runs exactly that configuration (bit-identical
to the explicit call)."""

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_TUNE = r"""
import sys, json
sys.path.insert(0, {root!r})
import torch
from paper_1710_01839_gb300 import inputs as I, tuner
A = torch.from_numpy(I.dd_random(384, 320, 61, 20)).cuda()
B = torch.from_numpy(I.dd_random(320, 448, 62, 20)).cuda()
C = torch.empty((2, 384, 448), dtype=torch.float64, device="cuda")
tuner.cache_open({path!r})
ch, rep = tuner.tune("dd", A, B, C, flags=tuner.REMEMBER | tuner.QUICK)
print(json.dumps([ch, rep["measured"], rep["from_cache"]]))
"""

_USE = r"""
import sys, json, ctypes
sys.path.insert(0, {root!r})
import numpy as np, torch
import paper_1710_01839_gb300 as mpg
from paper_1710_01839_gb300 import inputs as I, tuner
A = torch.from_numpy(I.dd_random(384, 320, 61, 20)).cuda()
B = torch.from_numpy(I.dd_random(320, 448, 62, 20)).cuda()
tuner.cache_open({path!r})
a, nm, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
assert mpg.lib().mpgemm_auto_choice(0, 0, 384, 320, 448, ctypes.byref(a), ctypes.byref(nm), ctypes.byref(d)) == 0
auto = mpg.gemm_dd(A, B, algo="auto").cpu().numpy()
name = {{0: "simple", 1: "block", 2: "strassen"}}[a.value]
explicit = mpg.gemm_dd(A, B, algo=name, n_min=nm.value, depth=d.value).cpu().numpy()
C = torch.empty((2, 384, 448), dtype=torch.float64, device="cuda")
ch, rep = tuner.tune("dd", A, B, C, flags=tuner.REMEMBER | tuner.QUICK)
print(json.dumps([[name, nm.value, d.value], bool(np.array_equal(auto, explicit)), ch, rep["measured"],
                  rep["from_cache"], tuner.cache_stats()]))
"""


def _py(code):
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    import json
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_auto_uses_choice_tuned_in_another_process(tmp_path):
    path = str(tmp_path / "tune.jsonl")
    ch, measured, from_cache = _py(_TUNE.format(root=ROOT, path=path))
    assert measured > 0 and not from_cache
    auto, same, ch2, measured2, from_cache2, stats = _py(_USE.format(root=ROOT, path=path))
    assert auto == [ch["algo"], ch["n_min"], ch["depth"]]
    assert same
    assert ch2 == ch and measured2 == 0 and from_cache2
    assert stats["choices"] == 1 and stats["measurements"] == measured and stats["skipped_lines"] == 0
