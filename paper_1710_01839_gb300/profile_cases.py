"""Fixed workloads for profiling: one GEMM configuration run a given number
of times on the seeded inputs of the benchmark workloads, so that an ncu
launch list or capture can be reproduced from the command line alone.

    python -m paper_1710_01839_gb300.profile_cases mp --bits 256 --n 512 --algo block --reps 2
    python -m paper_1710_01839_gb300.profile_cases mp --bits 128,256,512,1024 --n 256 --reps 2
    python -m paper_1710_01839_gb300.profile_cases split --fmt qd --n 1024 --reps 3
    python -m paper_1710_01839_gb300.profile_cases gemm --fmt qd --n 512 --algo block --n_min 32
    python -m paper_1710_01839_gb300.profile_cases via --fmt dd --bits 128 --n 2048 --algo strassen --n_min 512 --depth 3

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
    ap.add_argument("case", choices=["mp", "gemm", "split", "via"])
    ap.add_argument("--fmt", default="dd", choices=["dd", "qd"], help="gemm / split / via: element format")
    ap.add_argument("--bits", default="256", help="mp: precision(s) in bits, comma separated; via: limb precision")
    ap.add_argument("--n", type=int, default=512, help="m = l = n")
    ap.add_argument("--algo", default="block", choices=["simple", "block", "strassen"])
    ap.add_argument("--n_min", type=int, default=16)
    ap.add_argument("--depth", type=int, default=0)
    ap.add_argument("--slices", type=int, default=0, help="split: slice count (0 = the default)")
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args()

    import torch
    import paper_1710_01839_gb300 as mpg
    from paper_1710_01839_gb300 import inputs as I
    {"mp": _mp, "gemm": _gemm, "split": _split, "via": _via}[args.case](args, mpg, I, torch)
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main()
