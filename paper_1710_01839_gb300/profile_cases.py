"""Fixed workloads for profiling: one GEMM configuration run a given number
of times on the seeded inputs of the benchmark workloads, so that an ncu
launch list or capture can be reproduced from the command line alone.

    python -m paper_1710_01839_gb300.profile_cases mp --bits 256 --n 512 --algo block --reps 2
    python -m paper_1710_01839_gb300.profile_cases mp --bits 128,256,512,1024 --n 256 --reps 2
    python -m paper_1710_01839_gb300.profile_cases mp --bits 2048 --n 128 --leaf team --reps 2
    python -m paper_1710_01839_gb300.profile_cases leaves --bits 512,1024,2048 --shapes 32x32x32,16x4096x16
    python -m paper_1710_01839_gb300.profile_cases split --fmt qd --n 1024 --reps 3
    python -m paper_1710_01839_gb300.profile_cases gemm --fmt qd --n 512 --algo block --n_min 32
    python -m paper_1710_01839_gb300.profile_cases via --fmt dd --bits 128 --n 2048 --algo strassen --n_min 512 --depth 3

`leaves` times the block algorithm with the one-thread and the team
multi-limb kernels (CUDA events, best of 3 windows of 3 calls) and prints
one JSON line per shape.

Inputs: multi-limb mantissas uniform with exponents U{-64..64}
(inputs.mp_random, seeds 5 and 6); DD / QD entries with per-element
exponents 2^U{-20..20} (inputs.dd_random / qd_random); the DD split
workload's per-row and per-column spread 2^U{-16..16}
(inputs.dd_rowcol_scaled).  Prints "ok" after a device synchronize.
"""

from __future__ import annotations

import argparse


def _mp(args, mpg, I, torch):
    for bits in [int(b) for b in str(args.bits).split(",")]:
        w = bits // 32
        A = torch.from_numpy(I.mp_random(args.n, args.n, w, 5).view("int32")).cuda()
        B = torch.from_numpy(I.mp_random(args.n, args.n, w, 6).view("int32")).cuda()
        C = torch.empty_like(A)
        for _ in range(args.reps):
            mpg.gemm_mp(A, B, bits, C, algo=args.algo, n_min=args.n_min, depth=args.depth)


def _leaves(args, mpg, I, torch):
    import json
    shapes = [tuple(int(x) for x in s.split("x")) for s in args.shapes.split(",")]
    for bits in [int(b) for b in str(args.bits).split(",")]:
        w = bits // 32
        for m, l, n in shapes:
            A = torch.from_numpy(I.mp_random(m, l, w, 5).view("int32")).cuda()
            B = torch.from_numpy(I.mp_random(l, n, w, 6).view("int32")).cuda()
            C = torch.empty((2 + w, m, n), dtype=torch.int32, device="cuda")
            row = {"bits": bits, "m": m, "l": l, "n": n}
            for leaf in ("thread", "team"):
                mpg.set_mp_leaf(leaf)
                mpg.gemm_mp(A, B, bits, C, algo="block", n_min=16)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                best = float("inf")
                for _ in range(3):
                    e0.record()
                    for _ in range(3):
                        mpg.gemm_mp(A, B, bits, C, algo="block", n_min=16)
                    e1.record()
                    torch.cuda.synchronize()
                    best = min(best, e0.elapsed_time(e1) / 3)
                row[leaf + "_ms"] = round(best, 4)
            row["team_speedup"] = round(row["thread_ms"] / row["team_ms"], 3)
            print(json.dumps(row), flush=True)
    mpg.set_mp_leaf("default")


def _gemm(args, mpg, I, torch):
    gen = I.dd_random if args.fmt == "dd" else I.qd_random
    A = torch.from_numpy(gen(args.n, args.n, I.seed_for(1, 0), exp_spread=20)).cuda()
    B = torch.from_numpy(gen(args.n, args.n, I.seed_for(1, 1), exp_spread=20)).cuda()
    C = torch.empty_like(A)
    f = mpg.gemm_dd if args.fmt == "dd" else mpg.gemm_qd
    for _ in range(args.reps):
        f(A, B, C, algo=args.algo, n_min=args.n_min, depth=args.depth)


def _via(args, mpg, I, torch):
    gen = I.dd_random if args.fmt == "dd" else I.qd_random
    A = torch.from_numpy(gen(args.n, args.n, I.seed_for(1, 0), exp_spread=20)).cuda()
    B = torch.from_numpy(gen(args.n, args.n, I.seed_for(1, 1), exp_spread=20)).cuda()
    C = torch.empty_like(A)
    bits = int(str(args.bits).split(",")[0])
    for _ in range(args.reps):
        mpg.gemm_via_mp(A, B, bits, C, algo=args.algo, n_min=args.n_min, depth=args.depth)


def _split(args, mpg, I, torch):
    if args.fmt == "qd":
        A = I.qd_random(args.n, args.n, I.seed_for(1, 0), exp_spread=20)
        B = I.qd_random(args.n, args.n, I.seed_for(1, 1), exp_spread=20)
    else:
        A, B = I.dd_rowcol_scaled(args.n, args.n, args.n, seed=I.seed_for(3))
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    C = torch.empty_like(Ad)
    for _ in range(args.reps):
        mpg.gemm_split(Ad, Bd, C, slices=args.slices)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("case", choices=["mp", "gemm", "split", "via", "leaves"])
    ap.add_argument("--fmt", default="dd", choices=["dd", "qd"], help="gemm / split / via: element format")
    ap.add_argument("--bits", default="256", help="mp: precision(s) in bits, comma separated; via: limb precision")
    ap.add_argument("--n", type=int, default=512, help="m = l = n")
    ap.add_argument("--algo", default="block", choices=["simple", "block", "strassen"])
    ap.add_argument("--n_min", type=int, default=16)
    ap.add_argument("--depth", type=int, default=0)
    ap.add_argument("--slices", type=int, default=0, help="split: slice count (0 = the default)")
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--shapes", default="32x32x32,128x128x128,256x256x256",
                    help="leaves: m x l x n shapes, comma separated")
    ap.add_argument("--leaf", default="default", choices=["default", "thread", "team"],
                    help="mp: the block kernel at 512-2048 bits (mpgemm_set_mp_leaf)")
    args = ap.parse_args()

    import torch
    import paper_1710_01839_gb300 as mpg
    from paper_1710_01839_gb300 import inputs as I
    mpg.set_mp_leaf(args.leaf)
    {"mp": _mp, "gemm": _gemm, "split": _split, "via": _via, "leaves": _leaves}[args.case](args, mpg, I, torch)
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
