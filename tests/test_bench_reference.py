"""bench.py's reference arm (the oracle on the host cores) prints one JSON
line with every key of the benchmark contract (no GPU)."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("fmt", ["dd", "qd", "mp"])
def test_reference_arm_line(fmt):
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1", "--fmt", fmt,
           "--n", "64", "--cpu-seconds", "0.5", "--prec", "128"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["unit"] == "GFLOP/s" and d["higher_is_better"] is True
    assert d["dtype"] == ("u32" if fmt == "mp" else "f64")
    assert "m=l=n=64" in d["config"]["workload"]
    # the configuration the GPU arm's tuner picks at the benchmark sizes: the whole Strassen product
    assert (d["config"]["algo"], d["config"]["strassen_depth"]) == ("strassen", 4)
    assert "whole product" in d["cpu_baseline"]["sample"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
