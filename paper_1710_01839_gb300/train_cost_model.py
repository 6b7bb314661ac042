"""Train the FP32 MLP cost model on timings measured on this GPU and write it
to paper_1710_01839_gb300/data/cost_model_gb300.bin (or --out).

    python -m paper_1710_01839_gb300.train_cost_model [--count 5000] [--epochs 200]

Steps: mpgemm_cost_collect times `count` random configurations (shapes
log-uniform in [16, max_dim], DD / QD / 128- and 256-bit multi-limb, every valid
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
        for d in (1, 2, 3):
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
    args = ap.parse_args()
    import torch  # noqa: F401  (CUDA context, current stream)
    from paper_1710_01839_gb300 import costmodel as cm
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
