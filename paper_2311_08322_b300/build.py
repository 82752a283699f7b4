"""Build libgtb.so (all CUDA kernels + the C ABI) in-tree with nvcc for sm_103a,
and its checked twin libgtb_checked.so (the same sources compiled with
GTB_CHECKED: every kernel tests its address runs against the fields' storages and
reports a run outside them through gtb_device_status instead of touching it).

    python -m paper_2311_08322_b300.build [--force] [-v]
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libgtb.so")
LIB_CHECKED = os.path.join(PKG, "libgtb_checked.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-shared", "-cudart", "static",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def deps():
    return sources() + sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(ROOT, "include", "gtb.h")]


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in deps())


def _command(lib: str, verbose: bool):
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [NVCC, *ARCH, *FLAGS, *(["-DGTB_CHECKED"] if lib == LIB_CHECKED else []), "-o", tmp, *sources()]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    return cmd, tmp


def build(force: bool = False, verbose: bool = False, checked: bool = True) -> str:
    """Compile the libraries that are missing or older than their sources (both at once)."""
    libs = [LIB] + ([LIB_CHECKED] if checked else [])
    todo = [lib for lib in libs if force or stale(lib)]
    procs = []
    for lib in todo:
        cmd, tmp = _command(lib, verbose)
        procs.append((subprocess.Popen(cmd), tmp, lib))
    failed = [lib for p, _, lib in procs if p.wait() != 0]
    if failed:
        raise subprocess.CalledProcessError(1, "nvcc " + " ".join(os.path.basename(x) for x in failed))
    for _, tmp, lib in procs:
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
