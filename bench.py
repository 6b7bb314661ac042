#!/usr/bin/env python3
"""Benchmark of the multiple-precision GEMM C := AB on GB300.

One step = one C := AB at the large square configuration (DD by default,
m = l = n = 2048, entries hi ~ U[-1,1], lo = hi 2^-53 u, both words scaled
by 2^k, k ~ U{-20..20}) through the library's C ABI with the algorithm and
block size the tuner picked (the paper's Section 3 procedure: predict the
block algorithm's time for each n_min from a reduced-row run, then time
simple / block(best n_min) / Strassen and keep the fastest).  The tuning
itself runs once before the timed region and is reported, not timed.

Printed: one JSON line (rank 0).  `value` is whole-job effective GFLOP/s,
2 m n l / t (Strassen credited with the same nominal count), from CUDA
events on the launching stream with inputs resident in HBM and L2 flushed
between steps; `e2e` is the same metric with host->device copies of A and B
and the device->host copy of C inside the timed region.  `roofline` is the
dominant kernel's FP64-pipe utilisation (for multi-limb formats, its
integer issue rate); `cpu_baseline` is the oracle on the host cores over a
bounded row sample.

  python bench.py [--gpus N --steps K --warmup W] [--fmt dd|qd|mp [--prec BITS]] [--n 2048]
  python bench.py --impl reference ...   (the oracle on the host cores)
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "DD/QD GEMM GFLOP/s (2mnl/t) & roofline %; Ozaki vs plain DD at ≤2^-100 rel err"
# FP64-pipe operations per multiply-accumulate of the kernels (see ddqd.cuh;
# TwoSum's operand ordering runs on the integer pipe, and so does its error
# term except in the QD MAC's nine order-2 TwoSums: 1 FP64 operation per
# TwoSum, 3 for those nine; the DD MAC's product and its error run there too):
#   DD: 2 DFMA + TwoSum (1) + 2 DADD = 5, plus a 1-op TwoSum every 8 steps
#   QD: 50 per step (its six order-0..2 products through TwoProd on the
#       integer pipe) plus a 5-op renormalisation every 4 steps
FP64_OPS_PER_MAC = {"dd": 5.0 + 1.0 / 8.0, "qd": 50.0 + 5.0 / 4.0}
# FP64 pipe: 2 operations / clock / SM (measured 1.91 DFMA/clk/SM at 2.07 GHz by
# a dependent-chain-free DFMA loop) x 152 SMs x 2070 MHz maximum SM clock.
FP64_PEAK_GOPS = 2 * 152 * 2.070
# Issue rate: 1 warp-instruction / clock per SM sub-partition, 4 per SM.
ISSUE_PEAK_GWIPS = 4 * 152 * 2.070
# Multi-limb thread-instructions per multiply-accumulate (ncu
# smsp__inst_executed x 32 / MACs of the block kernel k_mp_block on 256^3
# (2048 bits: 128^3) inputs of the multi-limb workload), by precision in bits.
MP_INSTR_PER_MAC = {128: 232.2, 256: 376.7, 512: 963.6, 1024: 2610.1, 2048: 8472.3}
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the dominant
# kernel from ncu captures of exactly these configurations (profiles/),
# taken with the leaf kernel as it is now (entries of earlier forms of the
# kernel are dropped): (fmt, n, algo, n_min, depth) -> bytes.  Absent => null.
TRAFFIC_BYTES = {("dd", 2048, "strassen", 16, 4): 1.267e9 + 0.605e9}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mpgemm", choices=["mpgemm", "reference"])
    ap.add_argument("--fmt", default="dd", choices=["dd", "qd", "mp"])
    ap.add_argument("--prec", type=int, default=256, help="multi-limb precision in bits (--fmt mp)")
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--algo", default="tuned", choices=["tuned", "simple", "block", "strassen"])
    ap.add_argument("--n_min", type=int, default=64)
    ap.add_argument("--depth", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the split-precision comparison")
    ap.add_argument("--ozaki-n", type=int, default=4096)
    ap.add_argument("--ozaki-slices", type=int, default=16)
    ap.add_argument("--batched-count", type=int, default=512)
    ap.add_argument("--ozaki-fp8-slices", type=int, default=22)
    ap.add_argument("--qd-split-n", type=int, default=1024)
    ap.add_argument("--qd-split-slices", type=int, default=44)
    ap.add_argument("--extra-reps", type=int, default=5, help="timed calls (median) of each comparison arm")
    ap.add_argument("--no-peaks", action="store_true", help="use the fallback roofline peaks")
    ap.add_argument("--tuning-table", action="store_true",
                    help="run the Section 3 tuning-time experiment (paper_1710_01839_gb300.tuning_experiment) "
                         "over DD, QD and 128/256/1024-bit at n = 128..1024 +- 1 and print its JSON instead")
    return ap.parse_args()


# Roofline denominators.  Every run measures them itself with the library's
# peak microbenchmarks (mpgemm_peak_run, paper_1710_01839_gb300/peaks.py):
# tcgen05 e4m3 MMA, mma.sync s8, FP64 DFMA and 32-bit IMAD, each over about
# a second on every SM, with the SM clock sampled meanwhile.  The constants
# below are used only when that measurement is unavailable.
PEAKS = {}
PEAK_DESC = {"tc_e4m3": "tcgen05.mma kind::f8f6f4 M128 N256 K32, operands resident in shared memory",
             "mma_s8": "mma.sync m16n8k32 s8 on register operands",
             "fp64": "the fastest of FP64 DFMA, DADD and DMUL loops (independent chains, every SM full)",
             "imad": "mad.lo.u32, independent chains, every SM full"}


def _bf16x2_tflops():
    """The measured cuBLAS bf16 burst (MEASURED_PEAKS.json) x the nominal
    FP8 / BF16 ratio of 2 (fallback 1.9 PFLOP/s bf16)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return 2.0 * float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 2.0 * 1900.0


FALLBACK = {"tc_e4m3": (_bf16x2_tflops(), "fallback: measured cuBLAS bf16 burst x 2 (nominal FP8/BF16)"),
            "mma_s8": (151.2, "fallback: an earlier mma.sync s8 loop on this pool's GB300"),
            "fp64": (FP64_PEAK_GOPS, "fallback: derived 2 FP64 ops/clk/SM x 152 SMs x 2070 MHz"),
            "imad": (19.0, "fallback: an earlier IMAD loop on this pool's GB300")}


# The FP64 loop keeps the FP64 pipe busy 84.2 % of the time (ncu
# sm__pipe_fp64_cycles_active of k_peak_fp64<0>, profiles/peaks_microbenchmarks_gb300.md):
# the pipe's rate is the loop's measured rate / 0.842 (1.99 ops/clk/SM).
FP64_LOOP_PIPE_ACTIVE = 0.842


def peak(kind):
    """(value, note): this run's measured rate of `kind`, else the fallback."""
    p = PEAKS.get(kind)
    if p and kind == "fp64":
        v = p["value"] / FP64_LOOP_PIPE_ACTIVE
        return v, (f"measured in this run: the fastest FP64 loop ({p.get('source')}) ran {p['value']:.4g} G op/s at "
                   f"median SM clock {p['sm_mhz_median']} MHz with the FP64 pipe {FP64_LOOP_PIPE_ACTIVE:.1%} busy "
                   f"(ncu), so the pipe's rate is {v:.4g} G op/s")
    if p:
        src = f" ({p['source']})" if "source" in p else ""
        return p["value"], (f"measured in this run: {PEAK_DESC[kind]}{src}, {p['value']:.4g} {p['unit']} "
                            f"at median SM clock {p['sm_mhz_median']} MHz")
    return FALLBACK[kind]


def measure_peaks():
    try:
        from paper_1710_01839_gb300 import peaks
        PEAKS.update(peaks.measure_all(1.0))
    except Exception as e:   # reported, and the fallbacks are used
        PEAKS.clear()
        PEAKS["error"] = repr(e)


def timed_calls(fn, stream, reps=5, flush=None):
    """Median event time per call and median average duration of the
    dominant kernel's launches (the library's profiling brackets) over
    `reps` calls, after one untimed call; L2 flushed before every call."""
    import ctypes
    import torch
    import paper_1710_01839_gb300 as mpg
    L = mpg.lib()
    fn()
    torch.cuda.synchronize()
    ts, ks = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(reps):
        if flush is not None:
            flush.fill_(1.0)
        L.mpgemm_profile(1)
        L.mpgemm_profile_read(None, None)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        kms, kl = ctypes.c_double(), ctypes.c_int()
        L.mpgemm_profile_read(ctypes.byref(kms), ctypes.byref(kl))
        L.mpgemm_profile(0)
        ts.append(e0.elapsed_time(e1))
        ks.append(kms.value / max(kl.value, 1))
    return float(np.median(ts)), float(np.median(ks))


def _flush_buffer():
    import torch
    return torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")


def mp_roofline(bits, macs, k_ms, kname):
    """Multi-limb kernel: algorithmic IMAD fraction (2 w^2 32-bit IMADs per
    multiply-accumulate, the schoolbook limb products, against the measured
    IMAD rate) and the issue fraction of the instructions it executes."""
    w = bits // 32
    imad_peak, imad_note = peak("imad")
    alg = macs * 2.0 * w * w / (k_ms * 1e-3) / 1e12
    ipm = MP_INSTR_PER_MAC.get(bits)
    issue = macs * ipm / 32.0 / (k_ms * 1e-3) / 1e9 if ipm else None
    return {"bound": "alu", "unit": "T IMAD/s (algorithmic: 2 w^2 per MAC)", "achieved": alg, "peak": imad_peak,
            "frac": alg / imad_peak, "frac_algorithmic": alg / imad_peak, "peak_note": imad_note,
            "issue": {"unit": "G warp-instructions/s", "achieved": issue, "peak": ISSUE_PEAK_GWIPS,
                      "frac": issue / ISSUE_PEAK_GWIPS if issue else None, "instructions_per_mac": ipm,
                      "peak_note": "derived: 1 warp-instruction/clk per SM sub-partition x 4 x 152 SMs x 2070 MHz"},
            "kernel": f"{kname}, {macs:.3g} MACs x 2 w^2 = {2 * w * w} IMAD", "kernel_ms": k_ms}


def split_precision_extra(args, stream):
    """Ozaki-style split-precision DD GEMM against the plain DD kernels on the
    same DD inputs (m = l = n = ozaki_n, A's rows scaled by 2^r_i and B's
    columns by 2^c_j, r, c ~ U{-16..16}).  Accuracy (<= 2^-100 |A||B|) is
    asserted by the parity tests, not here."""
    import ctypes
    import torch
    import paper_1710_01839_gb300 as mpg
    from paper_1710_01839_gb300 import inputs as I
    n, S = args.ozaki_n, args.ozaki_slices
    A, B = I.dd_rowcol_scaled(n, n, n, seed=I.seed_for(3))
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    Cd = torch.empty_like(Ad)
    L = mpg.lib()
    sp = ctypes.c_void_p(int(stream.cuda_stream))
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    flush = _flush_buffer()
    reps = args.extra_reps

    def oz():
        rc = L.mpgemm_dd_ozaki(n, n, n, p(Ad), p(Bd), p(Cd), S, sp)
        if rc:
            raise RuntimeError(mpg.strerror(rc))

    flops = 2.0 * n ** 3
    oz_ms, oz_kms = timed_calls(oz, stream, reps, flush)
    pairs = S * (S + 1) // 2
    lp = (n + 127) // 128 * 128
    int_ops = 2.0 * n * n * lp * pairs
    s8_peak, s8_note = peak("mma_s8")
    out = {"workload": f"DD m=l=n={n}, rows/cols scaled 2^U{{-16..16}}, S={S} int8 slices",
           "timing": f"median of {reps} calls, L2 flushed (256 MB write) before each",
           "ozaki_gflops": flops / (oz_ms * 1e-3) / 1e9, "ozaki_ms": oz_ms,
           "roofline": {"bound": "tensor", "unit": "TOPS (int8 mma.sync)",
                        "achieved": int_ops / (oz_kms * 1e-3) / 1e12, "peak": s8_peak, "peak_note": s8_note,
                        "frac": int_ops / (oz_kms * 1e-3) / 1e12 / s8_peak,
                        "kernel": f"k_ozaki_levels, {pairs} slice pairs x 2 n^2 l int8 ops", "kernel_ms": oz_kms,
                        "kernel_share": oz_kms / oz_ms}}
    for name, algo, nm, d in (("plain_dd_block", "block", 64, 0), ("plain_dd_strassen4", "strassen", 32, 4)):
        ms, _ = timed_calls(lambda: mpg.gemm_dd(Ad, Bd, Cd, algo=algo, n_min=nm, depth=d), stream, reps, flush)
        out[name + "_gflops"] = flops / (ms * 1e-3) / 1e9
        out[name + "_ms"] = ms
    out["speedup_vs_best_plain_dd"] = min(out["plain_dd_block_ms"], out["plain_dd_strassen4_ms"]) / oz_ms
    # FP8 digits: balanced base-32, e4m3 tcgen05 MMAs with exact f32 accumulation in tensor memory
    S8 = args.ozaki_fp8_slices

    def oz8():
        rc = L.mpgemm_dd_ozaki_ex(n, n, n, p(Ad), p(Bd), p(Cd), S8, 1, sp)
        if rc:
            raise RuntimeError(mpg.strerror(rc))

    f8_ms, f8_kms = timed_calls(oz8, stream, reps, flush)
    pairs8 = S8 * (S8 + 1) // 2
    f8_flops = 2.0 * n * n * lp * pairs8
    out["fp8"] = {"slices": S8, "gflops": flops / (f8_ms * 1e-3) / 1e9, "ms": f8_ms,
                  "speedup_vs_int8": oz_ms / f8_ms,
                  "speedup_vs_best_plain_dd": min(out["plain_dd_block_ms"], out["plain_dd_strassen4_ms"]) / f8_ms,
                  "roofline": tc_roofline(f8_flops, f8_kms, f"k_levels_tc (tcgen05 kind::f8f6f4), {pairs8} slice "
                                                            "pairs x 2 n^2 l", f8_ms)}
    return out


def tc_roofline(flops, k_ms, kname, call_ms):
    tc_peak, tc_note = peak("tc_e4m3")
    ach = flops / (k_ms * 1e-3) / 1e12
    return {"bound": "tensor", "unit": "TFLOP/s (e4m3)", "achieved": ach, "peak": tc_peak, "peak_note": tc_note,
            "frac": ach / tc_peak, "frac_vs_bf16_burst_x2": ach / _bf16x2_tflops(), "kernel": kname,
            "kernel_ms": k_ms, "kernel_share": k_ms / call_ms}


def mlp_arm(fmt, Ad, Bd, Cd, gemm, tuned_ms, prec_bits):
    """The selection's third arm (the paper times every candidate; the
    prediction times samples; the FP32 MLP times nothing): the shipped cost
    model's choice, the host time of that decision, the choice's measured
    time and its regret against the tuned (measured) best."""
    import torch
    from paper_1710_01839_gb300 import costmodel
    if not os.path.exists(costmodel.DEFAULT_MODEL):
        return None
    costmodel.load(costmodel.DEFAULT_MODEL)
    m, l, n = Ad.shape[1], Ad.shape[2], Bd.shape[2]
    t0 = time.perf_counter()
    ch = costmodel.choice(fmt, m, l, n, prec_bits)
    decision_ms = (time.perf_counter() - t0) * 1e3
    if ch is None:
        return None
    run = lambda: gemm(Ad, Bd, Cd, algo=ch["algo"], n_min=ch["n_min"], depth=ch["depth"])
    run()
    torch.cuda.synchronize()
    times = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    return {"choice": {k: ch[k] for k in ("algo", "n_min", "depth")}, "predicted_ms": ch["pred_ms"],
            "measured_ms": ms, "regret_vs_tuned": ms / tuned_ms - 1.0, "decision_ms": decision_ms}


def qd_split_extra(args, stream):
    """Split-precision QD GEMM (FP8 digits of 4-term expansions, tcgen05)
    against the plain FP64-pipe QD kernels on the same QD inputs (the large
    QD workload: m = l = n = qd_split_n, per-element exponents 2^U{-20..20}).
    Accuracy (<= 4 l 2^-208 |A||B|) is asserted by the parity tests."""
    import torch
    import paper_1710_01839_gb300 as mpg
    n, S = args.qd_split_n, args.qd_split_slices
    A, B = inputs_for("qd", n)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    Cd = torch.empty_like(Ad)
    flush = _flush_buffer()
    reps = max(args.extra_reps, 10)

    flops = 2.0 * n ** 3
    sp_ms, sp_kms = timed_calls(lambda: mpg.gemm_split(Ad, Bd, Cd, slices=S), stream, reps, flush)
    lp = (n + 127) // 128 * 128
    tc_flops = 2.0 * n * n * lp * S * (S + 1) / 2
    out = {"workload": f"QD m=l=n={n}, per-element exponents 2^U{{-20..20}}, S={S} e4m3 slices",
           "timing": f"median of {reps} calls, L2 flushed (256 MB write) before each",
           "qd_split_gflops": flops / (sp_ms * 1e-3) / 1e9, "qd_split_ms": sp_ms,
           "roofline": tc_roofline(tc_flops, sp_kms, f"k_levels_tc (tcgen05 kind::f8f6f4), {S * (S + 1) // 2} "
                                                     "slice pairs x 2 n^2 l", sp_ms)}
    for name, algo, nm, d in (("plain_qd_block", "block", 32, 0), ("plain_qd_strassen4", "strassen", 16, 4)):
        ms, _ = timed_calls(lambda: mpg.gemm_qd(Ad, Bd, Cd, algo=algo, n_min=nm, depth=d), stream, args.extra_reps,
                            flush)
        out[name + "_gflops"] = flops / (ms * 1e-3) / 1e9
        out[name + "_ms"] = ms
    out["speedup_vs_best_plain_qd"] = min(out["plain_qd_block_ms"], out["plain_qd_strassen4_ms"]) / sp_ms
    return out


def via_mp_extra(args, stream, fp64_dd_gflops):
    """DD (at --n, 128-bit limbs) and QD (at --qd-split-n, 256-bit limbs)
    GEMMs on the integer pipe (mpgemm_dd_via_mp / mpgemm_qd_via_mp) on the
    same inputs as the FP64-pipe kernels: the multi-limb algorithm and n_min
    come from the Section 3 tuner run on the converted operands, and each
    timed call includes both conversions.  Accuracy (far inside the DD / QD
    bounds; bit-identical to the oracle) is asserted by the parity tests."""
    import torch
    import paper_1710_01839_gb300 as mpg
    from paper_1710_01839_gb300 import tuner
    out = {}
    flush = _flush_buffer()
    for fmt, n, bits, ref in (("dd", args.n, 128, fp64_dd_gflops), ("qd", args.qd_split_n, 256, None)):
        A, B = inputs_for(fmt, n)
        Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        Cd = torch.empty_like(Ad)
        Am, Bm = mpg.to_mp(Ad, bits), mpg.to_mp(Bd, bits)
        Cm = torch.empty_like(Am)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        choice, _ = tuner.tune("mp", Am, Bm, Cm, flags=tuner.QUICK, prec_bits=bits, stream=stream)
        t_tune = time.perf_counter() - t0
        del Am, Bm, Cm
        algo, n_min, depth = choice["algo"], choice["n_min"], choice["depth"]
        call = lambda: mpg.gemm_via_mp(Ad, Bd, bits, Cd, algo=algo, n_min=n_min, depth=depth, stream=stream)
        ms, k_ms = timed_calls(call, stream, args.extra_reps, flush)
        status = mpg.stream_status()
        if status != 0:
            raise RuntimeError(f"device status {status}: {mpg.strerror(status)}")
        flops = 2.0 * n ** 3
        leaf = (n + (1 << depth) - 1) >> depth if algo == "strassen" else n
        macs = (7 ** depth if algo == "strassen" else 1) * float(leaf) ** 3
        roof = mp_roofline(bits, macs, k_ms, f"{bits}-bit {'leaf ' if algo == 'strassen' else ''}GEMM")
        roof["kernel_share"] = k_ms / ms
        out[fmt] = {"workload": f"{fmt.upper()} m=l=n={n} (inputs of the FP64-pipe {fmt.upper()} GEMM), "
                                f"{bits}-bit limbs", "prec_bits": bits,
                    "timing": f"median of {args.extra_reps} calls, L2 flushed before each",
                    "choice": {"algo": algo, "n_min": n_min, "depth": depth}, "tuning_s": round(t_tune, 3),
                    "gflops": flops / (ms * 1e-3) / 1e9, "ms": ms, "roofline": roof}
        if ref is not None:
            out[fmt]["speedup_vs_fp64_pipe"] = out[fmt]["gflops"] / ref
    return out


def paper_matrices_extra(args, stream):
    """The paper's own workload (Section 4): A = [sqrt(5)(i+j-1)], B =
    [sqrt(3)(n-i)] at n = 1024 in DD and QD, each timed with the Section 3
    tuner's choice, and the largest relative error of sampled entries
    against the closed form c_ij = sqrt(15) n(n-1)(3i+n-2)/6 (sqrt(15) to
    300 bits)."""
    import math
    from fractions import Fraction
    import torch
    import paper_1710_01839_gb300 as mpg
    from paper_1710_01839_gb300 import inputs as I, tuner
    n = 1024
    r15 = Fraction(math.isqrt(15 << 600), 1 << 300)
    out = {"workload": f"Section 4 matrices A = sqrt(5)(i+j-1), B = sqrt(3)(n-i), n = {n}"}
    for fmt in ("dd", "qd"):
        A, B = I.paper_matrices(n, fmt)
        Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        Cd = torch.empty_like(Ad)
        torch.cuda.synchronize()
        choice, _ = tuner.tune(fmt, Ad, Bd, Cd, flags=tuner.QUICK, stream=stream)
        f = mpg.gemm_dd if fmt == "dd" else mpg.gemm_qd
        call = lambda: f(Ad, Bd, Cd, algo=choice["algo"], n_min=choice["n_min"], depth=choice["depth"], stream=stream)
        call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            call()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        C = Cd.cpu().numpy()
        worst = 0.0
        for i in (1, 2, n // 2, n):
            truth = r15 * I.paper_closed_form(n, i)
            for j in (0, n // 3, n - 1):
                got = sum((Fraction(float(C[t, i - 1, j])) for t in range(C.shape[0])), Fraction(0))
                worst = max(worst, float(abs(got - truth) / truth))
        out[fmt] = {"choice": choice, "gflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e9, "ms": ms,
                    "max_rel_err_vs_closed_form": worst}
    return out


def batched_extra(args, stream):
    """512 GEMMs, m, l, n log-uniform in [16, 1024], format uniform over
    {DD, QD, 256-bit}: one persistent graph-replayed launch with tiles from
    the FP32 MLP cost model, the same with tiles from exhaustive timing
    (every DD / QD GEMM timed alone at tile 16 and 32), and one ordinary
    launch per GEMM.  Effective GFLOP/s = 2 sum(m n l) / t."""
    import torch
    from paper_1710_01839_gb300 import batched, costmodel, inputs as I
    shapes = I.batched_shapes(args.batched_count)
    probs = []
    for i, (m, l, n, prec) in enumerate(shapes):
        s = I.seed_for(4, i)
        if prec == "dd":
            A, B, planes, dt = I.dd_random(m, l, s), I.dd_random(l, n, s + 1), 2, torch.float64
        elif prec == "qd":
            A, B, planes, dt = I.qd_random(m, l, s), I.qd_random(l, n, s + 1), 4, torch.float64
        else:
            A, B, planes, dt = I.mp_random(m, l, 8, s).view(np.int32), I.mp_random(l, n, 8, s + 1).view(np.int32), 10, torch.int32
        probs.append((prec, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                      torch.empty((planes, m, n), dtype=dt, device="cuda")))
    flops = 2.0 * sum(m * l * n for m, l, n, _ in shapes)
    model_src = "none"
    if os.path.exists(costmodel.DEFAULT_MODEL):
        costmodel.load(costmodel.DEFAULT_MODEL)
        model_src = "shipped model file (trained on this pool's GB300 by paper_1710_01839_gb300/train_cost_model.py)"
    else:
        F, T = costmodel.collect(2048, seed=1714, max_dim=1024)
        costmodel.train(F, T, epochs=200)
        model_src = "trained in this run on 2048 timings"

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    # exhaustive: each DD / QD GEMM alone at both tiles
    ex_tiles = []
    for prec, A, B, C in probs:
        if prec == "mp256":
            ex_tiles.append(16)
            continue
        one = batched.make_descs([(prec, A, B, C)], [16])
        t16 = timed(lambda: batched.sequential(one), 2)
        one[0].tile = 32
        t32 = timed(lambda: batched.sequential(one), 2)
        ex_tiles.append(16 if t16 < t32 else 32)
    d_model = batched.make_descs(probs)                 # tile 0: the cost model decides
    d_exh = batched.make_descs(probs, ex_tiles)
    p_model, p_exh = batched.Plan(d_model), batched.Plan(d_exh)
    t_model = timed(p_model.run_graph)
    t_exh = timed(p_exh.run_graph)
    t_seq = timed(lambda: batched.sequential(d_exh))
    model_tiles = p_model.info()["tiles"]
    p_model.close()
    p_exh.close()
    # the DD and QD GEMMs on the integer pipe (128 / 256-bit limbs, engine 1):
    # conversion passes + the persistent kernel in one graph, and one
    # mpgemm_*_via_mp launch per GEMM
    d_int = batched.make_descs(probs, integer_pipe=True)
    p_int = batched.Plan(d_int)
    t_int = timed(p_int.run_graph)
    t_int_seq = timed(lambda: batched.sequential(d_int))
    p_int.close()
    return {"workload": f"{len(shapes)} GEMMs, m,l,n log-uniform [16,1024], formats uniform over DD/QD/MP256",
            "persistent_graph_mlp_gflops": flops / (t_model * 1e-3) / 1e9, "persistent_graph_mlp_ms": t_model,
            "persistent_graph_exhaustive_gflops": flops / (t_exh * 1e-3) / 1e9, "persistent_graph_exhaustive_ms": t_exh,
            "sequential_launches_gflops": flops / (t_seq * 1e-3) / 1e9, "sequential_launches_ms": t_seq,
            "mlp_regret_vs_exhaustive": t_model / t_exh - 1, "persistent_speedup_vs_sequential": t_seq / t_exh,
            "tiles_agree_with_exhaustive": float(np.mean([a == b for a, b in zip(model_tiles, ex_tiles)])),
            "cost_model": model_src,
            "integer_pipe": {"persistent_graph_gflops": flops / (t_int * 1e-3) / 1e9, "persistent_graph_ms": t_int,
                             "sequential_launches_gflops": flops / (t_int_seq * 1e-3) / 1e9,
                             "sequential_launches_ms": t_int_seq,
                             "speedup_vs_fp64_persistent": t_model / t_int,
                             "note": "DD and QD GEMMs in 128 / 256-bit limbs (descriptor engine 1)"}}


# ---------------------------------------------------------------- helpers

def max_over_ranks(ms, dist=None, device="cpu"):
    """The slowest rank's time (replicas: every rank times its own GEMMs)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, flops_per_step, steps, t_max_ms):
    """Whole-job effective GFLOP/s: all ranks' nominal 2mnl work over the
    slowest rank's time."""
    return world * flops_per_step * steps / (t_max_ms * 1e-3) / 1e9


def inputs_for(fmt, n, rank=0, prec=256):
    from paper_1710_01839_gb300 import inputs as I
    if fmt == "mp":
        w = prec // 32
        A = I.mp_random(n, n, w, I.seed_for(2, 10 * rank + w))
        B = I.mp_random(n, n, w, I.seed_for(2, 10 * rank + w + 1))
        return A, B
    gen = I.dd_random if fmt == "dd" else I.qd_random
    A = gen(n, n, I.seed_for(1, 10 * rank), exp_spread=20)
    B = gen(n, n, I.seed_for(1, 10 * rank + 1), exp_spread=20)
    return A, B


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# The oracle's time for one whole Strassen product must stay a bounded
# sample of CPU work; above this estimate the CPU legs fall back to a row
# sample of the block algorithm (Strassen cannot be row-sampled).
STRASSEN_ORACLE_MAX_S = 20.0


def _oracle_run(fmt, A):
    import oracle
    if fmt == "mp":
        pb = 32 * (A.shape[0] - 2)
        return lambda A_, B_, **kw: oracle.mp_gemm(A_, B_, prec_bits=pb, **kw)
    return oracle.dd_gemm if fmt == "dd" else oracle.qd_gemm


def _oracle_strassen_fits(run, A, B, n_min, depth):
    """Estimate the oracle's time for the whole Strassen product: first from
    a few rows of its block algorithm (cheap, pessimistic up to about 3x:
    leaf work 7^d (n / 2^d)^3 of n^3); if that is within 4x of the limit,
    from the same Strassen call on the leading half-size problem (x 8)."""
    import oracle
    m, l, n = A.shape[1], A.shape[2], B.shape[2]
    rows = max(1, oracle.threads())
    t0 = time.perf_counter()
    run(A, B, algo="block", n_min=n_min, rows=(0, min(rows, m)))
    est = (time.perf_counter() - t0) * m / min(rows, m) * (7.0 / 8.0) ** depth
    if est <= STRASSEN_ORACLE_MAX_S:
        return True, est
    if est > 4 * STRASSEN_ORACLE_MAX_S:
        return False, est
    h = lambda x: max(2 ** depth, x // 2)
    Ah = np.ascontiguousarray(A[:, :h(m), :h(l)])
    Bh = np.ascontiguousarray(B[:, :h(l), :h(n)])
    t0 = time.perf_counter()
    run(Ah, Bh, algo="strassen", n_min=n_min, depth=depth)
    est = (time.perf_counter() - t0) * (m * l * n) / (h(m) * h(l) * h(n))
    return est <= STRASSEN_ORACLE_MAX_S, est


def cpu_baseline(fmt, A, B, algo, n_min, depth, budget_s):
    """The oracle (as it stands) on the host cores, on the configuration the
    GPU step runs: for Strassen the whole product at the same depth (when it
    fits the CPU budget), else a row sample of the block algorithm:
    rate = 2 * rows * n * l / t."""
    import oracle
    m, l, n = A.shape[1], A.shape[2], B.shape[2]
    run = _oracle_run(fmt, A)
    cores = oracle.threads()
    if algo == "strassen" and depth > 0:
        fits, est = _oracle_strassen_fits(run, A, B, n_min, depth)
        if fits:
            t0 = time.perf_counter()
            run(A, B, algo="strassen", n_min=n_min, depth=depth)
            dt = time.perf_counter() - t0
            return {"value": 2.0 * m * n * l / dt / 1e9, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                    "same_config": True,
                    "sample": f"the whole product ({fmt.upper()} Strassen depth {depth}, leaves block n_min {n_min}, "
                              f"the GPU step's configuration), {dt:.1f} s"}
    oalgo = "block" if algo in ("block", "strassen", "tuned") else "simple"
    rows = max(1, cores)
    t0 = time.perf_counter()
    run(A, B, algo=oalgo, n_min=n_min, rows=(0, rows))
    dt = time.perf_counter() - t0
    # grow the sample to about `budget_s` seconds in total
    if dt < budget_s / 4:
        more = int(rows * (budget_s * 0.75) / max(dt, 1e-3))
        more = max(rows, min(more - more % max(cores, 1), m - rows))
        t0 = time.perf_counter()
        run(A, B, algo=oalgo, n_min=n_min, rows=(rows, rows + more))
        dt = time.perf_counter() - t0
        rows = more
    gflops = 2.0 * rows * n * l / dt / 1e9
    return {"value": gflops, "unit": "GFLOP/s", "cores": cores, "kind": "oracle", "same_config": oalgo == algo,
            "sample": f"{rows} of {m} rows of C ({fmt.upper()} {oalgo} algorithm, k ascending), {dt:.1f} s"}


def workload_name(fmt, n, prec=256):
    """The benchmark workload, as both arms report it in `config`."""
    if fmt == "mp":
        return (f"{prec}-bit multi-limb square GEMM m=l=n={n}, uniform mantissa bits with the top bit set, "
                f"exponents U{{-64..64}}")
    lead = "hi~U[-1,1], lo=hi*2^-53*u" if fmt == "dd" else "x0~U[-1,1], x(i+1)=x(i)*2^-53*u(i)"
    return f"{fmt.upper()} square GEMM m=l=n={n}, {lead}, exponent spread 2^[-20,20]"


# ---------------------------------------------------------------- reference arm (the oracle)

# The configuration the reference arm times: what the Section 3 tuner picks
# on GB300 for the benchmark's DD 2048^3 workload (Strassen depth 4, n_min
# 32; the oracle's n_min only blocks its CPU loops, the arithmetic of every
# c_ij is the same at any n_min).
REF_ALGO, REF_N_MIN, REF_DEPTH = "strassen", 32, 4
REF_ARM_MAX_S = 300.0   # whole products for every step only while the run stays within this estimate


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    A, B = inputs_for(args.fmt, args.n, prec=args.prec)
    m, l, n = args.n, args.n, args.n
    run = _oracle_run(args.fmt, A)
    cores = oracle.threads()
    if args.algo == "tuned":
        algo, n_min, depth = REF_ALGO, REF_N_MIN, REF_DEPTH
    else:
        algo, n_min, depth = args.algo, args.n_min, args.depth if args.algo == "strassen" else 0
    if algo == "strassen" and depth > 0:
        fits, est = _oracle_strassen_fits(run, A, B, n_min, depth)
        if fits and est * (args.steps + args.warmup) <= REF_ARM_MAX_S:
            for _ in range(args.warmup):
                run(A, B, algo="strassen", n_min=n_min, depth=depth)
            times = []
            for _ in range(args.steps):
                t0 = time.perf_counter()
                run(A, B, algo="strassen", n_min=n_min, depth=depth)
                times.append(time.perf_counter() - t0)
            tot = sum(times)
            value = 2.0 * m * n * l * len(times) / tot / 1e9
            sample = (f"the whole product per step ({args.fmt.upper()} Strassen depth {depth}, leaves block "
                      f"n_min {n_min})")
            print(json.dumps(_reference_line(args, world, value, tot, len(times), cores, sample,
                                             {"algo": algo, "n_min": n_min, "strassen_depth": depth})), flush=True)
            return
    algo, depth = "block", 0
    per_step_rows = max(cores, 1)
    # size each step to about (cpu-seconds / 4) seconds
    t0 = time.perf_counter()
    run(A, B, algo="block", n_min=n_min, rows=(0, per_step_rows))
    dt = time.perf_counter() - t0
    target = max(1.0, args.cpu_seconds / 4)
    per_step_rows = int(min(m, max(per_step_rows, per_step_rows * target / max(dt, 1e-3))))
    for _ in range(args.warmup):        # untimed steps of the same size
        run(A, B, algo="block", n_min=n_min, rows=(0, per_step_rows))
    times = []
    for s in range(args.steps):
        r0 = (s * per_step_rows) % max(1, m - per_step_rows + 1)
        t0 = time.perf_counter()
        run(A, B, algo="block", n_min=n_min, rows=(r0, r0 + per_step_rows))
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = 2.0 * per_step_rows * n * l * len(times) / tot / 1e9
    sample = f"{per_step_rows} rows of C per step (of {m}), block algorithm"
    print(json.dumps(_reference_line(args, world, value, tot, len(times), cores, sample,
                                     {"algo": "block", "n_min": n_min, "strassen_depth": 0})), flush=True)


def _reference_line(args, world, value, tot_s, steps, cores, sample, cfg):
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32" if args.fmt == "mp" else "f64", "data": "synthetic",
            "config": dict({"workload": workload_name(args.fmt, args.n, args.prec), "fmt": args.fmt, "n": args.n},
                           **cfg),
            "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------- our arm

def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.tuning_table:
        from paper_1710_01839_gb300 import tuning_experiment
        print(json.dumps(tuning_experiment.run()), flush=True)
        return

    import torch
    import paper_1710_01839_gb300 as mpg
    from paper_1710_01839_gb300 import tuner

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    fmt, n = args.fmt, args.n
    m = l = n
    A, B = inputs_for(fmt, n, rank, args.prec)
    planes = A.shape[0]
    is_mp = fmt == "mp"
    Ad = torch.from_numpy(A.view(np.int32) if is_mp else A).cuda()
    Bd = torch.from_numpy(B.view(np.int32) if is_mp else B).cuda()
    Cd = torch.empty((planes, m, n), dtype=torch.int32 if is_mp else torch.float64, device="cuda")
    if is_mp:
        gemm = lambda A_, B_, C_, **kw: mpg.gemm_mp(A_, B_, args.prec, C_, **kw)
    else:
        gemm = mpg.gemm_dd if fmt == "dd" else mpg.gemm_qd

    # -------- selection (Section 3): untimed
    t_tune = 0.0
    tune_info = None
    if args.algo == "tuned":
        t0 = time.perf_counter()
        choice, tune_info = tuner.tune(fmt, Ad, Bd, Cd, flags=tuner.REMEMBER | tuner.VERIFY,
                                       prec_bits=args.prec if is_mp else 0)
        t_tune = time.perf_counter() - t0
        algo, n_min, depth = choice["algo"], choice["n_min"], choice["depth"]
        tune_info["mlp"] = mlp_arm(fmt, Ad, Bd, Cd, gemm, tune_info["best_ms"], args.prec if is_mp else 0)
    else:
        algo, n_min, depth = args.algo, args.n_min, args.depth if args.algo == "strassen" else 0

    def step():
        gemm(Ad, Bd, Cd, algo=algo, n_min=n_min, depth=depth)

    launches_per_step = 1 if algo in ("simple", "block") else 3 * depth + 1
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()
    L = mpg.lib()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # -------- timed region (device)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clk = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    L.mpgemm_profile(1)
    import ctypes
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    kms = ctypes.c_double(0.0)
    kl = ctypes.c_int(0)
    L.mpgemm_profile_read(ctypes.byref(kms), ctypes.byref(kl))
    L.mpgemm_profile(0)
    clocks = clk.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(step_ms)
    status = mpg.stream_status()
    if status != 0:
        raise RuntimeError(f"device status {status}: {mpg.strerror(status)}")
    t_max = max_over_ranks(tot_ms, dist, "cuda")
    flops_step = 2.0 * m * n * l
    value = whole_job_rate(world, flops_step, args.steps, t_max)

    # -------- end to end through host buffers
    e2e = None
    if not args.no_e2e:
        Ah = torch.from_numpy(A.view(np.int32) if is_mp else A).pin_memory()
        Bh = torch.from_numpy(B.view(np.int32) if is_mp else B).pin_memory()
        Ch = torch.empty((planes, m, n), dtype=Cd.dtype).pin_memory()
        for _ in range(2):
            Ad.copy_(Ah, non_blocking=True)
            Bd.copy_(Bh, non_blocking=True)
            step()
            Ch.copy_(Cd, non_blocking=True)
        torch.cuda.synchronize()
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(float(i))
            ev2[i][0].record(stream)
            Ad.copy_(Ah, non_blocking=True)
            Bd.copy_(Bh, non_blocking=True)
            step()
            Ch.copy_(Cd, non_blocking=True)
            ev2[i][1].record(stream)
        torch.cuda.synchronize()
        e_ms = sum(a.elapsed_time(b) for a, b in ev2)
        e_ms = max_over_ranks(e_ms, dist, "cuda")
        e2e = {"value": whole_job_rate(world, flops_step, args.steps, e_ms), "unit": "GFLOP/s",
               "h2d_bytes_per_step": int(A.nbytes + B.nbytes), "d2h_bytes_per_step": int(Ch.numel() * Ch.element_size()),
               "ms_per_step": e_ms / args.steps}

    # -------- roofline denominators, measured on this GPU (after the timed region)
    if not args.no_peaks:
        measure_peaks()

    # -------- dominant kernel roofline
    leaf = (n + (1 << depth) - 1) >> depth if algo == "strassen" else n
    leaf_count = 7 ** depth if algo == "strassen" else 1
    macs_per_launch = leaf_count * float(leaf) ** 3
    k_avg_ms = kms.value / max(kl.value, 1)
    kname = (f"{fmt} {'leaf ' if algo == 'strassen' else ''}{'simple' if algo == 'simple' else 'block'} GEMM")
    if is_mp:
        roofline = mp_roofline(args.prec, macs_per_launch, k_avg_ms, kname)
        roofline["traffic"] = None
    else:
        fp64_peak, fp64_note = peak("fp64")
        achieved = macs_per_launch * FP64_OPS_PER_MAC[fmt] / (k_avg_ms * 1e-3) / 1e9
        traffic = TRAFFIC_BYTES.get((fmt, n, algo, n_min, depth))
        roofline = {"bound": "alu", "unit": "Gop/s (FP64 pipe)", "achieved": achieved, "peak": fp64_peak,
                    "frac": achieved / fp64_peak, "traffic": traffic,
                    "kernel": f"{kname}, {macs_per_launch:.3g} MACs x {FP64_OPS_PER_MAC[fmt]} FP64 ops per launch",
                    "kernel_ms": k_avg_ms, "peak_note": fp64_note,
                    "frac_vs_derived_peak": achieved / FP64_PEAK_GOPS,
                    "derived_peak_note": "2 FP64 ops/clk/SM x 152 SMs x 2070 MHz = 629 G op/s"}
    roofline["kernel_share_of_step"] = kms.value / tot_ms if tot_ms else None

    extras = bextra = qextra = vextra = pextra = None
    if not args.no_extras and fmt == "dd":
        extras = split_precision_extra(args, stream)
        qextra = qd_split_extra(args, stream)
        vextra = via_mp_extra(args, stream, value / world)
        pextra = paper_matrices_extra(args, stream)
        if qextra is not None and "qd" in vextra:
            vextra["qd"]["speedup_vs_fp64_pipe"] = vextra["qd"]["gflops"] / max(qextra["plain_qd_block_gflops"],
                                                                                qextra["plain_qd_strassen4_gflops"])
        bextra = batched_extra(args, stream)

    if dist:
        dist.barrier()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    cpu = None
    if not args.no_cpu and world == 1:
        cpu = cpu_baseline(fmt, A, B, algo, n_min if n_min > 0 else 64, depth, args.cpu_seconds)

    line = {"metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32" if fmt == "mp" else "f64", "data": "synthetic",
            "config": {"workload": workload_name(fmt, n, args.prec), "fmt": fmt, "n": n, "algo": algo,
                       "n_min": n_min, "strassen_depth": depth, "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"replicas x{world}", "tuning_s": round(t_tune, 3)},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches_per_step * args.steps, "clocks": clocks}
    summary = {}
    if extras is not None:
        f8 = extras["fp8"]
        summary["dd_split_4096"] = {
            "int8_gflops": extras["ozaki_gflops"], "fp8_gflops": f8["gflops"],
            "plain_dd_block_gflops": extras["plain_dd_block_gflops"],
            "plain_dd_strassen4_gflops": extras["plain_dd_strassen4_gflops"],
            "fp8_speedup_vs_best_plain_dd": f8["speedup_vs_best_plain_dd"],
            "int8_speedup_vs_best_plain_dd": extras["speedup_vs_best_plain_dd"],
            "fp8_level_kernel_frac": f8["roofline"]["frac"], "int8_level_kernel_frac": extras["roofline"]["frac"]}
    if qextra is not None:
        summary["qd_split_1024"] = {"fp8_gflops": qextra["qd_split_gflops"],
                                    "speedup_vs_best_plain_qd": qextra["speedup_vs_best_plain_qd"],
                                    "level_kernel_frac": qextra["roofline"]["frac"]}
    if vextra is not None:
        summary["integer_pipe"] = {k: {"gflops": v["gflops"], "frac_algorithmic": v["roofline"]["frac_algorithmic"]}
                                   for k, v in vextra.items()}
    if PEAKS:
        summary["peaks"] = {k: (round(v["value"], 4) if isinstance(v, dict) else v) for k, v in PEAKS.items()
                            if k not in ("dfma", "dadd", "dmul")}
    if summary:
        line["summary"] = summary
    if PEAKS:
        line["peaks"] = PEAKS
    if tune_info is not None:
        line["tuning"] = tune_info
    if extras is not None:
        line["split_precision"] = extras
    if qextra is not None:
        line["qd_split_precision"] = qextra
    if vextra is not None:
        line["integer_pipe"] = vextra
    if pextra is not None:
        line["paper_matrices"] = pextra
    if bextra is not None:
        line["batched"] = bextra
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
