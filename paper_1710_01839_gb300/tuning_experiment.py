"""The tuning-time experiment of the paper's Section 3 and Tables 2 and 4, on
the GPU: for every format and size, the Section 3 procedure (mpgemm_tune)
is run with MPGEMM_TUNE_VERIFY, which times the block algorithm on the
reduced-row sample AND in full for every n_min.  From one run:

  * with prediction:    device time of the sampled runs + the final timings
                        (simple, block at the predicted n_min, Strassen 1..4);
  * without prediction: device time of the full block runs for every n_min
                        + the same final timings (the paper's exhaustive
                        alternative; it reports 1.6-2.3x more);
  * the FP32 MLP:       host time of its decision (nothing timed) and the
                        time of its pick against the tuned best, both with
                        the library's timer (mpgemm_time_config);
  * the fastest algorithm and, per format, the Strassen threshold: the
    smallest n from which Strassen is the fastest at every larger size
    (Table 2's "threshold" column).

    python -m paper_1710_01839_gb300.tuning_experiment [--formats dd,qd,mp128,mp256,mp1024] [--sizes 128,256,512,1024]

Sizes are n - 1, n, n + 1 for each n (the paper's Table 2).  Inputs: DD /
QD entries with per-element exponents 2^U{-20..20}, multi-limb mantissas
uniform with exponents U{-64..64} (the benchmark workloads).  Each
configuration is timed once after a warm-up run (MPGEMM_TUNE_QUICK).
Prints one JSON object.
"""

from __future__ import annotations

import argparse
import json
import time


def _operands(fmt, n, torch, I):
    if fmt == "dd":
        A, B = I.dd_random(n, n, 1710 + n, 20), I.dd_random(n, n, 1711 + n, 20)
    elif fmt == "qd":
        A, B = I.qd_random(n, n, 1710 + n, 20), I.qd_random(n, n, 1711 + n, 20)
    else:
        w = int(fmt[2:]) // 32
        A = I.mp_random(n, n, w, 1710 + n).view("int32")
        B = I.mp_random(n, n, w, 1711 + n).view("int32")
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    return Ad, Bd, torch.empty_like(Ad)


def run(formats=("dd", "qd", "mp128", "mp256", "mp1024"), sizes=(128, 256, 512, 1024)):
    import torch
    import paper_1710_01839_gb300 as mpg
    from paper_1710_01839_gb300 import costmodel, inputs as I, tuner
    have_model = False
    try:
        costmodel.load(costmodel.DEFAULT_MODEL)
        have_model = True
    except Exception:
        pass
    rows, thresholds = [], {}
    for fmt in formats:
        bits = int(fmt[2:]) if fmt.startswith("mp") else 0
        kind = "mp" if bits else fmt
        fastest = []
        for base in sizes:
            for n in (base - 1, base, base + 1):
                Ad, Bd, Cd = _operands(fmt, n, torch, I)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                choice, rep = tuner.tune(kind, Ad, Bd, Cd, flags=tuner.VERIFY | tuner.QUICK, prec_bits=bits)
                wall = time.perf_counter() - t0
                finals = [v for v in [rep["simple_ms"], rep["block_ms"]] + list(rep["strassen_ms"].values())
                          if v is not None]
                with_pred = sum(c["sample_ms"] for c in rep["candidates"]) + sum(finals)
                without = sum(c["full_ms"] for c in rep["candidates"]) + sum(finals)
                row = {"fmt": fmt, "n": n, "choice": choice, "best_ms": rep["best_ms"],
                       "device_ms_with_prediction": with_pred, "device_ms_without_prediction": without,
                       "cost_ratio_without_prediction": without / with_pred,
                       "max_prediction_rel_diff": rep.get("max_prediction_rel_diff"), "tuning_wall_s": wall}
                if have_model:
                    t1 = time.perf_counter()
                    mc = costmodel.choice(kind, n, n, n, prec_bits=bits)
                    dec_ms = (time.perf_counter() - t1) * 1e3
                    # both with the library's timer (calls back to back from C, the steady-state
                    # cost of a call, as MPGEMM_AUTO times): a timer in Python would add its own
                    # per-call overhead, a large share at these sizes
                    from paper_1710_01839_gb300.train_cost_model import _time_library
                    code = {"dd": 0, "qd": 1, "mp": 2}[kind]
                    t_mlp, t_best = _time_library(
                        code, bits, n, n, n, Ad, Bd, Cd,
                        [(mc["algo"], mc["n_min"], mc["depth"]), (choice["algo"], choice["n_min"], choice["depth"])])
                    row["mlp"] = {"choice": {k: mc[k] for k in ("algo", "n_min", "depth")},
                                  "decision_host_ms": dec_ms, "ms": t_mlp, "tuned_best_ms_same_session": t_best,
                                  "regret": t_mlp / t_best - 1}
                rows.append(row)
                fastest.append((n, choice["algo"]))
                del Ad, Bd, Cd
        # Table 2's threshold: Strassen fastest at this and every larger size
        thr = None
        for i in range(len(fastest)):
            if all(a == "strassen" for _, a in fastest[i:]):
                thr = fastest[i][0]
                break
        thresholds[fmt] = thr
    ratios = [r["cost_ratio_without_prediction"] for r in rows]
    return {"rows": rows, "strassen_threshold": thresholds,
            "cost_ratio_without_prediction": {"min": min(ratios), "max": max(ratios),
                                              "median": sorted(ratios)[len(ratios) // 2]},
            "total_device_s_with_prediction": sum(r["device_ms_with_prediction"] for r in rows) / 1e3,
            "total_device_s_without_prediction": sum(r["device_ms_without_prediction"] for r in rows) / 1e3,
            "note": "device times are one timed run per configuration (QUICK); the warm-up run before each "
                    "doubles both totals alike"}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--formats", default="dd,qd,mp128,mp256,mp1024")
    ap.add_argument("--sizes", default="128,256,512,1024")
    a = ap.parse_args()
    res = run(tuple(a.formats.split(",")), tuple(int(x) for x in a.sizes.split(",")))
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
