"""The paper's thread-count axis on a GPU.

Section 4 times every algorithm with 1, 2, 4 and 8 OpenMP threads and
reports, per size and thread count, the fastest algorithm and the block
size n_min the prediction picked (Tables 1-4).  Here the same procedure
(mpgemm_tune: predicted n_min from row-sampled runs, then simple, block and
Strassen depths 1-4 timed) runs on SM partitions holding 1/8, 1/4, 1/2 and
all of the device's SMs, on square DD, QD and 256-bit problems with the
inputs of the large DD/QD and multi-limb workloads.

    python -m paper_1710_01839_gb300.partition_sweep [--out sweep.json]
    python -m paper_1710_01839_gb300.partition_sweep --precisions [--out map.json]
    python -m paper_1710_01839_gb300.partition_sweep --paper-tables [--out tables.json]

prints one markdown table and optionally writes the rows as JSON; with
--precisions it maps the fastest algorithm and the tuning time over the
multi-limb precisions 128..2048 bits (the paper's Figure 2 and Table 4);
with --paper-tables it gives the rows of the paper's Tables 1 and 3 (n =
1024; DD, QD, 128- and 1024-bit multi-limb for MPFR 128 / 1024 bits; the
SM partitions for 1, 2, 4, 8 threads): the predicted n_min, the block and
the best Strassen time, and the prediction against the full block run.
"""

from __future__ import annotations

import argparse
import json


def _inputs(fmt, n, seed):
    """fmt: "dd", "qd", "mp" (256 bits) or "mpNNN" (NNN bits)."""
    import numpy as np
    from . import inputs as I
    if fmt == "dd":
        return I.dd_random(n, n, seed, 20), I.dd_random(n, n, seed + 1, 20), 0
    if fmt == "qd":
        return I.qd_random(n, n, seed, 20), I.qd_random(n, n, seed + 1, 20), 0
    bits = int(fmt[2:]) if len(fmt) > 2 else 256
    A, B = I.mp_random(n, n, bits // 32, seed), I.mp_random(n, n, bits // 32, seed + 1)
    return A.view(np.int32), B.view(np.int32), bits


def sweep(fractions=(8, 4, 2, 1), sizes=None, flags=None):
    import torch
    from . import Partition, tuner
    sizes = sizes or {"dd": (128, 256, 512, 1024, 1025), "qd": (128, 256, 512), "mp": (128, 256, 512)}
    flags = tuner.QUICK if flags is None else flags
    total = torch.cuda.get_device_properties(0).multi_processor_count
    rows = []
    for frac in fractions:
        want = max(1, total // frac)
        part = Partition(want) if frac > 1 else None
        stream = part.stream if part else torch.cuda.current_stream()
        sms = part.sms if part else total
        try:
            for fmt, ns in sizes.items():
                for n in ns:
                    A, B, bits = _inputs(fmt, n, 1710 + n)
                    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
                    Cd = torch.empty_like(Ad)
                    torch.cuda.synchronize()
                    choice, rep = tuner.tune(fmt, Ad, Bd, Cd, flags=flags, prec_bits=bits, stream=stream)
                    rows.append({"sms": sms, "fmt": fmt if fmt != "mp" else "mp256", "n": n,
                                 "algo": choice["algo"], "n_min": choice["n_min"], "depth": choice["depth"],
                                 "best_ms": rep["best_ms"], "simple_ms": rep["simple_ms"],
                                 "block_ms": rep["block_ms"], "strassen_ms": rep["strassen_ms"],
                                 "gflops": 2.0 * n ** 3 / (rep["best_ms"] * 1e-3) / 1e9})
        finally:
            if part:
                part.close()
    return rows


def paper_tables(fractions=(8, 4, 2, 1), formats=("dd", "qd", "mp128", "mp1024"), n=1024):
    """Tables 1 and 3 of the paper on SM partitions: for every format and
    partition, the Section 3 procedure with every n_min's full block run as
    well (VERIFY), so the prediction of the chosen n_min can be compared
    with its measured time (the paper's last two columns)."""
    import torch
    from . import Partition, tuner
    total = torch.cuda.get_device_properties(0).multi_processor_count
    rows = []
    for frac in fractions:
        part = Partition(max(1, total // frac)) if frac > 1 else None
        stream = part.stream if part else torch.cuda.current_stream()
        sms = part.sms if part else total
        try:
            for fmt in formats:
                A, B, bits = _inputs(fmt, n, 1710 + n)
                Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
                Cd = torch.empty_like(Ad)
                torch.cuda.synchronize()
                kind = "mp" if fmt.startswith("mp") else fmt
                choice, rep = tuner.tune(kind, Ad, Bd, Cd, flags=tuner.QUICK | tuner.VERIFY | tuner.SKIP_SIMPLE,
                                         prec_bits=bits, stream=stream)
                best_pred = min(rep["candidates"], key=lambda c: c["pred_ms"])
                st = {d: v for d, v in rep["strassen_ms"].items() if v is not None}
                d_best = min(st, key=st.get) if st else None
                flop = 2.0 * n ** 3
                rows.append({"sms": sms, "fmt": fmt, "n": n, "n_min": best_pred["n_min"],
                             "block_ms": rep["block_ms"], "block_gflops": flop / (rep["block_ms"] * 1e-3) / 1e9,
                             "strassen_depth": d_best, "strassen_ms": st.get(d_best),
                             "strassen_gflops": flop / (st[d_best] * 1e-3) / 1e9 if st else None,
                             "pred_ms": best_pred["pred_ms"], "full_ms": best_pred["full_ms"],
                             "rel_diff": best_pred["rel_diff"], "fastest": choice["algo"],
                             "fastest_depth": choice["depth"]})
                del Ad, Bd, Cd
        finally:
            if part:
                part.close()
    return rows


def paper_table(rows):
    lines = ["| format | SMs | n_min (predicted) | block ms (GFLOP/s) | best Strassen ms (GFLOP/s) | predicted ms | "
             "rel. diff |", "|---|---|---|---|---|---|---|"]
    for r in rows:
        stv = "-" if r["strassen_ms"] is None else \
            f"d={r['strassen_depth']}: {r['strassen_ms']:.4g} ({r['strassen_gflops']:.3g})"
        lines.append(f"| {r['fmt']} | {r['sms']} | {r['n_min']} | {r['block_ms']:.4g} ({r['block_gflops']:.3g}) | "
                     f"{stv} | {r['pred_ms']:.4g} | {100 * r['rel_diff']:.2f} % |")
    return "\n".join(lines)


def precision_sweep(precisions=(128, 256, 512, 1024, 2048), sizes=(128, 256, 512, 1024), max_2048=512):
    """The paper's multi-precision map (its Figure 2 and Table 4): for every
    multi-limb precision and size, the tuner's fastest algorithm, its time
    and the tuner's own wall time, on the whole device (2048 bits up to
    max_2048, its runs being long)."""
    import numpy as np
    import time
    import torch
    from . import inputs as I
    from . import tuner
    rows = []
    for bits in precisions:
        for n in sizes:
            if bits == 2048 and n > max_2048:
                continue
            w = bits // 32
            A = I.mp_random(n, n, w, 1710 + n).view(np.int32)
            B = I.mp_random(n, n, w, 1711 + n).view(np.int32)
            Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
            Cd = torch.empty_like(Ad)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            choice, rep = tuner.tune("mp", Ad, Bd, Cd, flags=tuner.QUICK, prec_bits=bits)
            wall = time.perf_counter() - t0
            rows.append({"bits": bits, "n": n, "algo": choice["algo"], "n_min": choice["n_min"],
                         "depth": choice["depth"], "best_ms": rep["best_ms"], "tuning_s": wall,
                         "gflops": 2.0 * n ** 3 / (rep["best_ms"] * 1e-3) / 1e9})
    return rows


def precision_table(rows):
    lines = ["| bits | n | fastest | n_min | best ms | GFLOP/s | tuning s |", "|---|---|---|---|---|---|---|"]
    for r in rows:
        algo = r["algo"] + (f" d={r['depth']}" if r["algo"] == "strassen" else "")
        lines.append(f"| {r['bits']} | {r['n']} | {algo} | {r['n_min']} | {r['best_ms']:.3g} | {r['gflops']:.3g} | "
                     f"{r['tuning_s']:.2f} |")
    return "\n".join(lines)


def table(rows):
    lines = ["| SMs | format | n | fastest | n_min | best ms | GFLOP/s | simple / block / Strassen d=1,2,3,4 ms |",
             "|---|---|---|---|---|---|---|---|"]
    for r in rows:
        st = r["strassen_ms"]
        others = " / ".join("-" if v is None else f"{v:.3g}"
                            for v in [r["simple_ms"], r["block_ms"], st.get(1), st.get(2), st.get(3), st.get(4)])
        algo = r["algo"] + (f" d={r['depth']}" if r["algo"] == "strassen" else "")
        lines.append(f"| {r['sms']} | {r['fmt']} | {r['n']} | {algo} | {r['n_min']} | {r['best_ms']:.3g} | "
                     f"{r['gflops']:.3g} | {others} |")
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", default=None, help="write the rows as JSON here")
    ap.add_argument("--precisions", action="store_true",
                    help="instead: the multi-limb precision map (128..2048 bits) on the whole device")
    ap.add_argument("--paper-tables", action="store_true",
                    help="instead: the rows of the paper's Tables 1 and 3 (n = 1024) on the SM partitions")
    args = ap.parse_args()
    if args.paper_tables:
        rows = paper_tables()
        print(paper_table(rows))
    elif args.precisions:
        rows = precision_sweep()
        print(precision_table(rows))
    else:
        rows = sweep()
        print(table(rows))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(rows, f, indent=1)


if __name__ == "__main__":
    main()
