"""Build the CUDA library ``libvr.so`` in-tree (nvcc, sm_103a only).

Usage: ``python -m paper_1205_0282_gb300.build [--verbose]``.  The library
exports the C ABI declared in ``include/vr.h``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libvr.so")
SOURCES = ["vr_host.cu", "vr_kernels.cu", "vr_march_tma.cu", "vr_march_tex.cu", "vr_noalloc.cu", "vr_shard.cu", "vr_ooc.cu", "vr_serve.cu", "vr_codec.cu"]
HEADERS = ["df.cuh", "vr_blocks.h", "vr_internal.cuh", "vr_device.cuh", "vr_alpha_fit.h", "vr_ctx.cuh", "tc.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "vr.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=PKG)
    os.close(fd)
    cmd = [nvcc(), "-O3", "-std=c++17", *ARCH, "-lineinfo", "--threads", "0",
           "-Xcompiler", "-fPIC", "-shared", "-o", tmp,
           *[os.path.join(CSRC, f) for f in SOURCES]]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd), flush=True)
    try:
        subprocess.run(cmd, check=True)
    except BaseException:
        if os.path.exists(tmp):
            os.remove(tmp)
        raise
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="--verbose" in sys.argv)
    print(LIB)
