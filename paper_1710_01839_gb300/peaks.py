"""Measured peak rates of the instructions the library's kernels are bound
by (the roofline denominators), from the library's own microbenchmarks
(mpgemm_peak_run): tcgen05 e4m3 MMA, mma.sync s8, FP64 DFMA, DADD and DMUL
(the FP64 pipe's rate, "fp64", is the fastest of the three) and 32-bit
IMAD.

    python -m paper_1710_01839_gb300.peaks [--seconds 1.0]

Each rate is operations / second over a timed region of about `seconds`
(CUDA events on the launching stream, after one untimed launch), with the
SM clock sampled by nvidia-smi during the region; `per_clk_per_sm` divides
by the median sampled clock and the SM count, and `at_max_clock` scales the
rate to the maximum SM clock.
"""

from __future__ import annotations

import ctypes
import json
import statistics
import subprocess
import threading

KINDS = {"tc_e4m3": 0, "mma_s8": 1, "dfma": 2, "imad": 3, "dadd": 4, "dmul": 5}
UNITS = {"tc_e4m3": "TFLOP/s", "mma_s8": "TOPS", "dfma": "G FP64 op/s", "imad": "T thread-IMAD/s",
         "dadd": "G FP64 op/s", "dmul": "G FP64 op/s"}
SCALE = {"tc_e4m3": 1e12, "mma_s8": 1e12, "dfma": 1e9, "imad": 1e12, "dadd": 1e9, "dmul": 1e9}
# iterations per launch: a few to some tens of milliseconds each
ITERS = {"tc_e4m3": 1 << 14, "mma_s8": 1 << 14, "dfma": 1 << 12, "imad": 1 << 15, "dadd": 1 << 12, "dmul": 1 << 12}


class _Clocks:
    def __init__(self, idx=0):
        self.idx, self.proc, self.sm, self.mx = idx, None, [], []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=clocks.sm,clocks.max.sm",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            f = [x.strip() for x in ln.split(",")]
            try:
                self.sm.append(float(f[0]))
                self.mx.append(float(f[1]))
            except (ValueError, IndexError):
                pass

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=5)


def measure(name: str, seconds: float = 1.0, stream=None) -> dict:
    import torch
    import paper_1710_01839_gb300 as mpg
    L = mpg.lib()
    stream = stream or torch.cuda.current_stream()
    sp = ctypes.c_void_p(int(stream.cuda_stream))
    ops = ctypes.c_double()
    iters = ITERS[name]

    def launch():
        rc = L.mpgemm_peak_run(KINDS[name], iters, ctypes.byref(ops), sp)
        if rc:
            raise RuntimeError(f"mpgemm_peak_run({name}): {mpg.strerror(rc)}")

    launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launch()
    e1.record(stream)
    torch.cuda.synchronize()
    one_ms = max(e0.elapsed_time(e1), 1e-3)
    launches = max(3, int(seconds * 1e3 / one_ms))
    with _Clocks() as clk:
        e0.record(stream)
        for _ in range(launches):
            launch()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    if mpg.stream_status() != 0:
        raise RuntimeError(f"peak loop {name}: device status set")
    rate = ops.value * launches / (ms * 1e-3)
    sms = L.mpgemm_stream_sms(sp)
    mhz = statistics.median(clk.sm) if clk.sm else None
    mx = max(clk.mx) if clk.mx else None
    out = {"value": rate / SCALE[name], "unit": UNITS[name], "ms": ms, "launches": launches,
           "sm_mhz_median": mhz, "sm_max_mhz": mx, "clock_samples": len(clk.sm)}
    if mhz:
        out["per_clk_per_sm"] = rate / (mhz * 1e6) / sms
        if mx:
            out["at_max_clock"] = rate * mx / mhz / SCALE[name]
    return out


def measure_all(seconds: float = 1.0, stream=None) -> dict:
    out = {k: measure(k, seconds * (2.0 if k == "tc_e4m3" else (0.5 if k in ("dadd", "dmul") else 1.0)), stream)
           for k in KINDS}
    # the FP64 pipe: the fastest of the DFMA, DADD and DMUL loops
    best = max(("dfma", "dadd", "dmul"), key=lambda k: out[k]["value"])
    out["fp64"] = dict(out[best], source=best)
    return out


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--seconds", type=float, default=1.0)
    ap.add_argument("--kind", default="all", choices=["all"] + list(KINDS))
    a = ap.parse_args()
    res = measure_all(a.seconds) if a.kind == "all" else {a.kind: measure(a.kind, a.seconds)}
    print(json.dumps(res, indent=1))
