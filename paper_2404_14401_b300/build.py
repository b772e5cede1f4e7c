"""Build the sm_103a CUDA library libgpe.so in-tree (nvcc, no GPU needed).

Each .cu file is compiled to an object in parallel (separate nvcc processes;
gpe_kernels.cu in KERNEL_PARTS parts, each emitting a share of the kernel
instantiations), then the objects are linked into the shared library.  No relocatable device
code: the files share no device functions.
"""
from __future__ import annotations

import concurrent.futures
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = [os.path.join(HERE, "csrc", f) for f in ("gpe_api.cu", "gpe_kernels.cu", "gpe_batch.cu", "gpe_static.cu",
                                                       "gpe_pair.cu", "gpe_coop.cu")]
DEPS = SRC + [os.path.join(HERE, "csrc", f) for f in ("gpe_fft.cuh", "gpe_fft2.cuh", "gpe_device.cuh", "gpe_internal.h",
                                                       "gpe_pair.cuh", "gpe_ctrl.cuh")] + [
    os.path.join(os.path.dirname(HERE), "include", "gpe.h")]
LIB = os.path.join(HERE, "libgpe.so")
DEBUG_LIB = os.path.join(HERE, "libgpe_debug.so")  # -DGPE_DEBUG_BOUNDS=1: index checks that latch GPE_EBOUNDS
OBJDIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-diag-suppress", "128"]
KERNEL_PARTS = 5                                   # parts of gpe_kernels.cu compiled side by side


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in DEPS)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile libgpe.so for sm_103a if missing or older than its sources;
    debug=True: the bounds-check build libgpe_debug.so (-DGPE_DEBUG_BOUNDS=1),
    whose kernels check their global indices and shared-memory regions and
    latch GPE_EBOUNDS instead of making an out-of-bounds access."""
    lib = DEBUG_LIB if debug else LIB
    objdir = os.path.join(OBJDIR, "debug") if debug else OBJDIR
    if force or stale(lib):
        os.makedirs(objdir, exist_ok=True)
        flags = [*ARCH, *FLAGS] + (["-DGPE_DEBUG_BOUNDS=1"] if debug else []) + (["-Xptxas=-v"] if verbose else [])
        jobs = []                                   # (source, object, extra flags)
        for f in SRC:
            base = os.path.basename(f)[:-3]
            if base == "gpe_kernels":               # compiled in parts (GPE_PART in the file)
                jobs += [(f, os.path.join(objdir, f"{base}_p{k}.o"), [f"-DGPE_PART={k}"]) for k in range(KERNEL_PARTS)]
            else:
                jobs.append((f, os.path.join(objdir, base + ".o"), []))
        objs = [o for _, o, _ in jobs]
        with concurrent.futures.ThreadPoolExecutor(len(jobs)) as ex:
            runs = [ex.submit(subprocess.run, [nvcc(), *flags, *x, "-c", f, "-o", o], check=True)
                    for f, o, x in jobs]
            for r in runs:
                r.result()
        tmp = lib + ".tmp"
        subprocess.run([nvcc(), *ARCH, "-shared", *objs, "-o", tmp], check=True)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))
