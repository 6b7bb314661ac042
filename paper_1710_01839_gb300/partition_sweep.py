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

prints one markdown table and optionally writes the rows as JSON; with
--precisions it maps the fastest algorithm and the tuning time over the
multi-limb precisions 128..2048 bits (the paper's Figure 2 and Table 4).
"""

from __future__ import annotations

import argparse
import json


def _inputs(fmt, n, seed):
    import numpy as np
    from . import inputs as I
    if fmt == "dd":
        return I.dd_random(n, n, seed, 20), I.dd_random(n, n, seed + 1, 20), 0
    if fmt == "qd":
        return I.qd_random(n, n, seed, 20), I.qd_random(n, n, seed + 1, 20), 0
    A, B = I.mp_random(n, n, 8, seed), I.mp_random(n, n, 8, seed + 1)
    return A.view(np.int32), B.view(np.int32), 256


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
    args = ap.parse_args()
    if args.precisions:
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
