"""The C ABI is usable from plain C (no GPU): include/mpgemm.h compiles as
C99, and a C program linked against libmpgemm.so calls the host-only entry
points and gets argument errors back before any device call."""

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "mpgemm.h"

int main(void) {
    /* negative sizes: refused before anything touches a device */
    int rc_dd = mpgemm_dd(-1, 4, 4, NULL, NULL, NULL, MPGEMM_BLOCK, 0, 0, NULL);
    int rc_mp = mpgemm_mp(4, -1, 4, 128, NULL, NULL, NULL, MPGEMM_BLOCK, 0, 0, NULL);
    size_t ws_block = mpgemm_workspace_size(MPGEMM_KIND_DD, 0, 64, 64, 64, MPGEMM_BLOCK, 0);
    size_t ws_str = mpgemm_workspace_size(MPGEMM_KIND_DD, 0, 64, 64, 64, MPGEMM_STRASSEN, 1);
    printf("%d %d %d %zu %d %s|%s\n", mpgemm_version() >= 100, rc_dd, rc_mp, ws_block, ws_str > 0,
           mpgemm_strerror(MPGEMM_OK), mpgemm_strerror(MPGEMM_EINVAL));
    return 0;
}
"""


def test_header_is_c99_and_a_c_program_links_and_runs(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_1710_01839_gb300 import build
    build.build()
    libdir = os.path.join(ROOT, "paper_1710_01839_gb300", "_build")
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                    "-L", libdir, "-lmpgemm", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")      # a host-only run, whatever the machine
    out = subprocess.run([str(exe)], capture_output=True, text=True, env=env, check=True).stdout.strip()
    assert out == "1 -1 -1 0 1 ok|invalid argument", out
