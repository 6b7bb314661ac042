"""The persistent tuning cache (mpgemm_tune_cache_open) with a simulated
timer (mpgemm_tune_set_timer), no GPU: the Section 3 procedure runs on
deterministic fake timings, its timings and choice go to an append-only
JSON-lines file, a second process reads them back (choice answered without
timing, MPGEMM_AUTO uses it), a run killed mid-way resumes without timing
again what it had finished and ends with the uninterrupted run's choice,
and damaged or foreign lines are skipped."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tuner():
    from paper_1710_01839_gb300 import build
    build.build()
    from paper_1710_01839_gb300 import tuner as t
    return t


def fake_ms(kind, bits, m, l, n, algo, n_min, depth, rows, reps):
    """A cost model with a clear optimum: block best at n_min 64, Strassen
    depth 2 fastest overall (7/8 of the work per level, plus overhead)."""
    base = 1e-6 * rows * l * n
    penalty = 1.0 + 0.05 * abs((n_min.bit_length() - 1) - 6)
    if algo == 0:
        return 3.0 * base
    if algo == 1:
        return base * penalty
    return base * penalty * (7 / 8) ** depth + 0.02 * depth * depth * base


_CHILD = r"""
import os, sys
sys.path.insert(0, {root!r})
from paper_1710_01839_gb300 import tuner
sys.path.insert(0, os.path.join({root!r}, "tests"))
from test_tune_cache import fake_ms
calls = [0]
def timer(*a):
    calls[0] += 1
    if calls[0] > {kill_after}:
        os._exit(17)          # killed mid-run: no clean-up, no final record
    return fake_ms(*a)
tuner.cache_open({path!r})
tuner.set_timer(timer)
rep = tuner.tune_shape("dd", 4096, 256, 4096, flags=tuner.REMEMBER | tuner.VERIFY)
print("finished", rep["measured"])
"""


def _child(path, kill_after):
    code = _CHILD.format(root=ROOT, path=str(path), kill_after=kill_after)
    return subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300, cwd=ROOT)


def _counting(counter):
    def timer(*a):
        counter.append(a)
        return fake_ms(*a)
    return timer


def _run(tuner, path, shape=(4096, 256, 4096), flags=None):
    flags = tuner.REMEMBER | tuner.VERIFY if flags is None else flags
    calls = []
    tuner.cache_open(path)
    tuner.set_timer(_counting(calls))
    try:
        rep = tuner.tune_shape("dd", *shape, flags=flags)
    finally:
        tuner.set_timer(None)
        tuner.cache_open(None)
    return rep, calls


def test_round_trip_and_auto(tuner, tmp_path):
    path = tmp_path / "tune.jsonl"
    tuner.lib().mpgemm_tune_forget()
    rep, calls = _run(tuner, path)
    # 6 sampled + 6 full block runs (VERIFY), simple, Strassen d = 1..4 (at
    # m = n = 4096 every sample has fewer rows than the full run; the final
    # block run at the chosen n_min is the VERIFY run of the same configuration)
    assert rep["measured"] == len(calls) == 6 + 6 + 1 + 4
    assert not rep["from_cache"]
    assert (rep["algo"], rep["n_min"], rep["depth"]) == ("strassen", 64, 2)
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert [x["t"] for x in lines].count("meas") == len(calls)
    assert [x["t"] for x in lines].count("choice") == 1 and lines[-1]["t"] == "choice"
    # a second process: the choice comes from the file, nothing is timed, AUTO uses it
    code = (f"import sys, ctypes; sys.path.insert(0, {ROOT!r})\n"
            "from paper_1710_01839_gb300 import tuner\n"
            f"tuner.cache_open({str(path)!r})\n"
            "print(tuner.cache_stats())\n"
            "a, nm, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()\n"
            "assert tuner.lib().mpgemm_auto_choice(0, 0, 4096, 256, 4096, ctypes.byref(a), ctypes.byref(nm), "
            "ctypes.byref(d)) == 0\n"
            "print('auto', a.value, nm.value, d.value)\n"
            "tuner.set_timer(lambda *x: 1 / 0)\n"
            "r = tuner.tune_shape('dd', 4096, 256, 4096)\n"
            "print('again', r['from_cache'], r['measured'], r['algo'], r['n_min'], r['depth'])\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    out = r.stdout.splitlines()
    stats = eval(out[0])
    assert stats["choices"] == 1 and stats["measurements"] == len(calls) and stats["skipped_lines"] == 0
    assert out[1] == "auto 2 64 2"
    assert out[2] == "again True 0 strassen 64 2"
    # the file is unchanged by a cached answer
    assert len(path.read_text().splitlines()) == len(lines)


def test_killed_run_resumes(tuner, tmp_path):
    full, full_calls = _run(tuner, tmp_path / "reference.jsonl")
    path = tmp_path / "tune.jsonl"
    kill_after = 7
    r = _child(path, kill_after)
    assert r.returncode == 17, (r.returncode, r.stdout, r.stderr[-2000:])
    kinds = [json.loads(x)["t"] for x in path.read_text().splitlines()]
    assert kinds == ["meas"] * kill_after            # every finished timing, no choice
    rep, calls = _run(tuner, path)
    assert rep["measured"] == len(calls) == len(full_calls) - kill_after
    assert not rep["from_cache"]
    for k in ("algo", "n_min", "depth", "best_ms", "block_ms"):
        assert rep[k] == full[k]
    assert [c["pred_ms"] for c in rep["candidates"]] == [c["pred_ms"] for c in full["candidates"]]
    # the resumed run timed exactly the configurations the killed one had not reached
    done = set(full_calls[:kill_after])
    assert not done & set(calls) and set(full_calls) == done | set(calls)


def test_damaged_and_foreign_lines_are_skipped(tuner, tmp_path):
    path = tmp_path / "tune.jsonl"
    _run(tuner, path)
    good = path.read_text()
    first = json.loads(good.splitlines()[0])
    foreign = dict(first, dev="Some Other GPU")
    old = dict(first, ver=1)
    damaged = (good
               + "not json at all\n"
               + '{"v":1,"t":"meas","dev":"x"}\n'            # missing fields
               + '{"v":2,"t":"meas"}\n'                       # unknown version of the format
               + json.dumps(foreign).replace(" ", "") + "\n"
               + json.dumps(old).replace(" ", "") + "\n"
               + '{"v":1,"t":"choice","dev":')                # cut short, no newline
    path.write_text(damaged)
    tuner.cache_open(path)
    try:
        st = tuner.cache_stats()
        assert st["open"] and st["choices"] == 1 and st["measurements"] == 17
        assert st["skipped_lines"] == 4 and st["foreign_records"] == 2
        calls = []
        tuner.set_timer(_counting(calls))
        rep = tuner.tune_shape("dd", 256, 512, 384)     # another shape: tuned and appended
        assert rep["measured"] == len(calls) > 0
    finally:
        tuner.set_timer(None)
        tuner.cache_open(None)
    lines = path.read_text().split("\n")
    # the cut-short line was ended before the new records; every new line parses
    tail = lines[len(damaged.split("\n")):]
    assert tail[-1] == "" and all(json.loads(x)["m"] == 256 for x in tail[:-1])
    assert json.loads(tail[-2])["t"] == "choice"


def test_force_retunes_from_cached_timings(tuner, tmp_path):
    path = tmp_path / "tune.jsonl"
    first, _ = _run(tuner, path)
    rep, calls = _run(tuner, path, flags=tuner.REMEMBER | tuner.VERIFY | tuner.FORCE)
    assert not rep["from_cache"] and rep["measured"] == 0 and not calls
    assert (rep["algo"], rep["n_min"], rep["depth"]) == (first["algo"], first["n_min"], first["depth"])
    # without VERIFY the procedure needs no full block runs: all in the cache too
    rep, calls = _run(tuner, path, flags=tuner.FORCE)
    assert rep["measured"] == 0 and not calls


def test_cache_arguments(tuner, tmp_path):
    L = tuner.lib()
    assert L.mpgemm_tune_cache_open(b"") == -1
    assert L.mpgemm_tune_cache_open(os.fsencode(tmp_path / "no" / "such" / "dir" / "f")) == -1
    assert L.mpgemm_tune_cache_open(None) == 0
    assert tuner.cache_stats()["open"] is False
    with pytest.raises(RuntimeError):
        tuner.tune_shape("dd", 64, 64, 64)       # no timer set: refuses to pass placeholder operands
