"""Train the FP32 MLP cost model on timings measured on this GPU and write it
to paper_1710_01839_gb300/data/cost_model_gb300.bin (or --out).

    python -m paper_1710_01839_gb300.train_cost_model [--count 5000] [--epochs 200]

Steps: mpgemm_cost_collect times `count` random configurations (shapes
log-uniform in [16, max_dim], DD / QD / 128- to 1024-bit multi-limb, every valid
algorithm / tile / Strassen depth); 90 % train the model (mpgemm_cost_train),
10 % measure its held-out error.  Then, for a set of random shapes, the
configuration the library's choice rule picks with the model
(mpgemm_cost_choice) is timed against every candidate timed exhaustively,
and the regret (t_model / t_best - 1) is reported.  Prints one JSON report.
--evaluate MODEL runs only the regret study of a saved model.
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
if os.path.dirname(HERE) not in sys.path:
    sys.path.insert(0, os.path.dirname(HERE))


def _time(fn, reps=3):
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def _time_interleaved(fns, reps=5, window_ms=1.0):
    """Steady-state ms per call of each function: calls issued back to back
    between two events, enough of them to fill about `window_ms` (at most
    20), the windows of all functions timed round-robin `reps` times (round
    r of every function before round r + 1 of any); median over rounds."""
    import torch
    counts = []
    for f in fns:
        f()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        f()
        b.record()
        torch.cuda.synchronize()
        counts.append(max(1, min(20, int(window_ms / max(a.elapsed_time(b), 1e-3)))))
    ts = [[] for _ in fns]
    for _ in range(reps):
        for i, f in enumerate(fns):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            for _ in range(counts[i]):
                f()
            b.record()
            torch.cuda.synchronize()
            ts[i].append(a.elapsed_time(b) / counts[i])
    return [float(np.median(t)) for t in ts]


def _time_library(kind, bits, m, l, n, Ad, Bd, Cd, cands, reps=5):
    """Each candidate (algo, n_min, depth) timed with the library's own timer
    (mpgemm_time_config: calls back to back between two events, from C, as
    MPGEMM_AUTO times its short list), 10 / 3 / 1 calls per window for
    candidates below 1 / 20 ms / above, windows round-robin over the
    candidates `reps` times; median over rounds."""
    import ctypes
    import paper_1710_01839_gb300 as mpg
    L = mpg.lib()
    codes = {"simple": 0, "block": 1, "strassen": 2}
    p = lambda t: ctypes.c_void_p(t.data_ptr())

    def one(c, r):
        ms = ctypes.c_double()
        rc = L.mpgemm_time_config(kind, bits, m, l, n, p(Ad), p(Bd), p(Cd), codes[c[0]], c[1], c[2], r, None,
                                  ctypes.byref(ms))
        if rc:
            raise RuntimeError(f"mpgemm_time_config: {mpg.strerror(rc)}")
        return ms.value

    calls = []
    for c in cands:
        t = one(c, 1)
        calls.append(10 if t < 1.0 else 3 if t < 20.0 else 1)
    ts = [[] for _ in cands]
    for _ in range(reps):
        for i, c in enumerate(cands):
            ts[i].append(one(c, calls[i]))
    return [float(np.median(t)) for t in ts]


def batched_like_shapes(count, seed=2024, min_dim=16, max_dim=1024):
    """(fmt, bits, m, l, n): m, l, n log-uniform in [min_dim, max_dim] (the
    batched workload's recipe), formats cycling DD, QD, 256-bit, 128-bit."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        fmt, bits = [("dd", 0), ("qd", 0), ("mp", 256), ("mp", 128)][i % 4]
        m, l, n = (int(round(x)) for x in np.exp(rng.uniform(np.log(min_dim), np.log(max_dim), 3)))
        out.append((fmt, bits, m, l, n))
    return out


def auto_regret_study(shapes, reps=5):
    """MPGEMM_AUTO's pick (the cost model, with its short list timed on the
    operands when the model is not sure) against every candidate timed
    exhaustively with the library's timer (_time_library), one GEMM at a
    time; also the model's pick alone."""
    import ctypes
    import torch
    import paper_1710_01839_gb300 as mpg
    from paper_1710_01839_gb300 import costmodel as cm, inputs as I
    L = mpg.lib()
    rows = []
    for i, (fmt, bits, m, l, n) in enumerate(shapes):
        if fmt == "dd":
            A, B = I.dd_random(m, l, 500 + i), I.dd_random(l, n, 600 + i)
        elif fmt == "qd":
            A, B = I.qd_random(m, l, 500 + i), I.qd_random(l, n, 600 + i)
        else:
            A, B = I.mp_random(m, l, bits // 32, 500 + i), I.mp_random(l, n, bits // 32, 600 + i)
        Ad = torch.from_numpy(A.view(np.int32) if fmt == "mp" else A).cuda()
        Bd = torch.from_numpy(B.view(np.int32) if fmt == "mp" else B).cuda()

        def run(algo, tile, depth):
            if fmt == "dd":
                return lambda: mpg.gemm_dd(Ad, Bd, algo=algo, n_min=tile, depth=depth)
            if fmt == "qd":
                return lambda: mpg.gemm_qd(Ad, Bd, algo=algo, n_min=tile, depth=depth)
            return lambda: mpg.gemm_mp(Ad, Bd, bits, algo=algo, n_min=tile, depth=depth)

        tmax = {"dd": 64, "qd": 32, "mp": 16}[fmt]
        ext = lambda x, d: (x + (1 << d) - 1) >> d << d
        cands = [("simple", 16, 0)] + [("block", t, 0) for t in (16, 32, 64) if t <= tmax]
        for d in (1, 2, 3, 4):
            if all((ext(x, d) >> d) >= 16 for x in (m, l, n)):
                cands += [("strassen", t, d) for t in (16, 32, 64) if t <= tmax]
        kind = {"dd": 0, "qd": 1, "mp": 2}[fmt]
        L.mpgemm_tune_forget()
        run("auto", 0, 0)()                                 # AUTO decides (and remembers)
        torch.cuda.synchronize()
        a, nm, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check = L.mpgemm_auto_choice(kind, bits, m, l, n, ctypes.byref(a), ctypes.byref(nm), ctypes.byref(d))
        assert check == 0
        auto = ({0: "simple", 1: "block", 2: "strassen"}[a.value], nm.value, d.value)
        ch = cm.choice(fmt, m, l, n, prec_bits=bits)        # the model's rule alone (nothing timed)
        rule = (ch["algo"], ch["n_min"], ch["depth"])
        for c in (auto, rule):
            if c not in cands:
                cands.append(c)
        Cd = torch.empty((Ad.shape[0], m, n), dtype=Ad.dtype, device="cuda")
        meas = _time_library(kind, bits, m, l, n, Ad, Bd, Cd, cands, reps)
        best = int(np.argmin(meas))
        t_auto, t_rule = meas[cands.index(auto)], meas[cands.index(rule)]
        rows.append({"fmt": fmt if fmt != "mp" else f"mp{bits}", "m": m, "l": l, "n": n, "auto_pick": auto,
                     "model_rule_pick": rule, "best": cands[best], "t_auto_ms": t_auto, "t_rule_ms": t_rule,
                     "t_best_ms": meas[best], "regret_auto": t_auto / meas[best] - 1,
                     "regret_model_rule": t_rule / meas[best] - 1})
        del Ad, Bd
    L.mpgemm_tune_forget()
    ra = [r["regret_auto"] for r in rows]
    rr = [r["regret_model_rule"] for r in rows]
    return {"shapes": rows, "count": len(rows),
            "auto": {"mean": float(np.mean(ra)), "median": float(np.median(ra)), "max": float(np.max(ra)),
                     "over_10pct": int(np.sum(np.array(ra) > 0.10)),
                     "time_weighted": float(sum(r["t_auto_ms"] for r in rows) / sum(r["t_best_ms"] for r in rows) - 1)},
            "model_rule": {"mean": float(np.mean(rr)), "median": float(np.median(rr)), "max": float(np.max(rr)),
                           "over_10pct": int(np.sum(np.array(rr) > 0.10))}}


def regret_study(shapes_seed=99, count=12, max_dim=1024):
    """Model's pick vs exhaustive timing of all candidates, single GEMMs."""
    import torch
    import paper_1710_01839_gb300 as mpg
    from paper_1710_01839_gb300 import costmodel as cm, inputs as I
    rng = np.random.default_rng(shapes_seed)
    rows = []
    for i in range(count):
        fmt, bits = [("dd", 0), ("qd", 0), ("mp", 256), ("mp", 128)][i % 4]
        dims = [int(x) // 8 * 8 for x in np.exp(rng.uniform(np.log(64), np.log(max_dim), 3))]
        m, l, n = (max(d, 16) for d in dims)
        if fmt == "dd":
            A, B = I.dd_random(m, l, i), I.dd_random(l, n, i + 1)
        elif fmt == "qd":
            A, B = I.qd_random(m, l, i), I.qd_random(l, n, i + 1)
        else:
            A, B = I.mp_random(m, l, bits // 32, i), I.mp_random(l, n, bits // 32, i + 1)
        Ad = torch.from_numpy(A.view(np.int32) if fmt == "mp" else A).cuda()
        Bd = torch.from_numpy(B.view(np.int32) if fmt == "mp" else B).cuda()

        def run(algo, tile, depth):
            if fmt == "dd":
                return lambda: mpg.gemm_dd(Ad, Bd, algo=algo, n_min=tile, depth=depth)
            if fmt == "qd":
                return lambda: mpg.gemm_qd(Ad, Bd, algo=algo, n_min=tile, depth=depth)
            return lambda: mpg.gemm_mp(Ad, Bd, bits, algo=algo, n_min=tile, depth=depth)

        tmax = {"dd": 64, "qd": 32, "mp": 16}[fmt]
        cands = [("simple", 16, 0)] + [("block", t, 0) for t in (16, 32, 64) if t <= tmax]
        for d in (1, 2, 3, 4):
            if all(x % (1 << d) == 0 and (x >> d) >= 16 for x in (m, l, n)):
                cands += [("strassen", t, d) for t in (16, 32, 64) if t <= tmax]
        ch = cm.choice(fmt, m, l, n, prec_bits=bits)      # the library's rule (mpgemm_cost_choice)
        pick_c = (ch["algo"], ch["n_min"], ch["depth"])
        if pick_c not in cands:
            cands.append(pick_c)
        pick = cands.index(pick_c)
        meas = [_time(run(*c)) for c in cands]
        best = int(np.argmin(meas))
        rows.append({"fmt": fmt if fmt != "mp" else f"mp{bits}", "m": m, "l": l, "n": n, "model_pick": cands[pick], "best": cands[best],
                     "t_model_ms": meas[pick], "t_best_ms": meas[best], "regret": meas[pick] / meas[best] - 1,
                     "pred_ms_of_pick": float(ch["pred_ms"])})
    reg = [r["regret"] for r in rows]
    return {"shapes": rows, "mean_regret": float(np.mean(reg)), "median_regret": float(np.median(reg)),
            "max_regret": float(np.max(reg))}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=5000)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--max-dim", type=int, default=1024)
    ap.add_argument("--seed", type=int, default=1714)
    ap.add_argument("--out", default=None)
    ap.add_argument("--regret-shapes", type=int, default=12)
    ap.add_argument("--evaluate", default=None, metavar="MODEL",
                    help="only load MODEL and run the regret study (no collection or training)")
    ap.add_argument("--auto-regret", type=int, default=0, metavar="SHAPES",
                    help="with --evaluate: MPGEMM_AUTO's regret on SHAPES shapes drawn like the batched workload")
    args = ap.parse_args()
    import torch  # noqa: F401  (CUDA context, current stream)
    from paper_1710_01839_gb300 import costmodel as cm
    if args.evaluate and args.auto_regret:
        cm.load(args.evaluate)
        print(json.dumps({"model": args.evaluate,
                          "auto_regret": auto_regret_study(batched_like_shapes(args.auto_regret))}), flush=True)
        return
    if args.evaluate:
        cm.load(args.evaluate)
        print(json.dumps({"model": args.evaluate,
                          "regret": regret_study(count=args.regret_shapes, max_dim=args.max_dim)}), flush=True)
        return
    t0 = time.time()
    F, T = cm.collect(args.count, seed=args.seed, max_dim=args.max_dim)
    t_collect = time.time() - t0
    ntr = int(0.9 * len(T)) // 128 * 128
    t0 = time.time()
    loss = cm.train(F[:ntr], T[:ntr], epochs=args.epochs, seed=args.seed)
    t_train = time.time() - t0
    pred = cm.predict(F[ntr:])
    rel = np.abs(pred / T[ntr:] - 1)
    out = args.out or cm.DEFAULT_MODEL
    cm.save(out)
    report = {"samples": int(len(T)), "train": ntr, "heldout": int(len(T) - ntr), "collect_s": t_collect,
              "train_s": t_train, "loss_first": float(loss[0]), "loss_last": float(loss[-1]),
              "heldout_median_rel_err": float(np.median(rel)), "heldout_p90_rel_err": float(np.quantile(rel, 0.9)),
              "heldout_within_25pct": float(np.mean(rel < 0.25)), "model": out}
    if args.regret_shapes > 0:
        report["regret"] = regret_study(count=args.regret_shapes, max_dim=args.max_dim)
    print(json.dumps(report), flush=True)


if __name__ == "__main__":
    main()
