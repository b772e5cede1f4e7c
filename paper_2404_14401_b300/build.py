"""Build the sm_103a CUDA library libgpe.so in-tree (nvcc, no GPU needed)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = [os.path.join(HERE, "csrc", f) for f in ("gpe_api.cu", "gpe_kernels.cu", "gpe_static.cu")]
DEPS = SRC + [os.path.join(HERE, "csrc", f) for f in ("gpe_fft.cuh", "gpe_internal.h")] + [
    os.path.join(os.path.dirname(HERE), "include", "gpe.h")]
LIB = os.path.join(HERE, "libgpe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
         "-diag-suppress", "128"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libgpe.so for sm_103a if missing or older than its sources."""
    if force or stale():
        cmd = [nvcc(), *ARCH, *FLAGS, *SRC, "-o", LIB]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
