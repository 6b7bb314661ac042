"""Build libmpgemm.so (all CUDA sources, sm_103a) in-tree.

    python -m paper_1710_01839_gb300.build        # or __graft_entry__.build()

Each translation unit is compiled by nvcc in parallel, then linked into
paper_1710_01839_gb300/_build/libmpgemm.so (shared CUDA runtime, so the
library and PyTorch share one runtime and one context).  The same sources
compiled with -DMPGEMM_BOUNDS_CHECK give the bounds-checked build,
_build_bc/libmpgemm_bc.so (a testing tool: every global access of the GEMM
kernels checked against its buffer), built alongside in the same pool.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libmpgemm.so")
OUT_BC = os.path.join(HERE, "_build_bc")
LIB_BC = os.path.join(OUT_BC, "libmpgemm_bc.so")
# (output folder, library, extra nvcc flags)
VARIANTS = [(OUT, LIB, []), (OUT_BC, LIB_BC, ["-DMPGEMM_BOUNDS_CHECK"])]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "--fmad=false", "-Xcompiler", "-fPIC,-O2",
                     "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps_newer(target: str) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    files = glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(ROOT, "include", "*.h"))
    return any(os.path.getmtime(f) > t for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    """Build both variants (each only if a source is newer); returns the
    product library's path."""
    todo = [v for v in VARIANTS if force or _deps_newer(v[1])]
    if not todo:
        return LIB
    cc = nvcc()
    for out, _, _ in todo:
        os.makedirs(out, exist_ok=True)

    def compile_one(job):
        (out, _, extra), src = job
        obj = os.path.join(out, os.path.basename(src)[:-3] + ".o")
        cmd = [cc] + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)} {' '.join(extra)}:\n{r.stderr}")
        return obj

    # the product's translation units first, the longest first within each
    jobs = [(v, src) for v in todo for src in sorted(sources(), key=lambda f: -os.path.getsize(f))]
    workers = min(len(jobs), max(2, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(compile_one, jobs))
    for out, lib, extra in todo:
        mine = [o for o in objs if os.path.dirname(o) == out]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [cc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + mine
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
