"""Compile the CUDA sources into the in-tree shared library libhplmm.so (sm_103a).

Usage: python -m paper_2509_19777_gb300.build   (or call build_library()).
Each translation unit is compiled in parallel with nvcc, then linked with the
static CUDA runtime into one C-ABI shared object beside this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libhplmm.so")
STAMP = OUT + ".sha256"
BUILD_DIR = os.path.join(HERE, "_build")
SOURCES = ["prims.cu", "assemble.cu", "maps.cu", "local.cu", "coarse.cu", "cfactor.cu", "apply.cu", "capi.cu", "static_spmv.cu",
           "checkpoint.cu", "ilu.cu",
           "ws.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc():
    exe = shutil.which("nvcc")
    if exe is None:
        cand = "/usr/local/cuda/bin/nvcc"
        if os.path.exists(cand):
            exe = cand
    if exe is None:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhplmm.so")
    return exe


def _compile(src, extra):
    obj = os.path.join(BUILD_DIR, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def source_hash():
    """SHA-256 over the sources, headers, compiler flags and this machine's architecture: the identity of a
    build.  A library copied from another machine or built from other sources never matches it."""
    h = hashlib.sha256()
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h")))
    files.append(os.path.join(os.path.dirname(HERE), "include", "hplmm.h"))
    for p in files:
        h.update(os.path.basename(p).encode())
        with open(p, "rb") as f:
            h.update(f.read())
    h.update(" ".join(ARCH + FLAGS).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def build_library(verbose=False, ptxas_info=False, force=False):
    """Build libhplmm.so unless the library beside this file was built from exactly these sources on this
    kind of machine (a hash of them is recorded next to it), or always when force is set."""
    want = source_hash()
    if not force and os.path.exists(OUT) and os.path.exists(STAMP):
        with open(STAMP) as f:
            if f.read().strip() == want:
                return OUT
    os.makedirs(BUILD_DIR, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    if verbose or ptxas_info:
        for obj, log in results:
            if log.strip():
                print(f"== {os.path.basename(obj)}\n{log}", file=sys.stderr)
    tmp = OUT + ".tmp"
    # -ldl: the NVTX 3 header loads a profiler's injection library with dlopen (in libc from glibc 2.34 on)
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *[o for o, _ in results], "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, OUT)
    with open(STAMP, "w") as f:
        f.write(want + "\n")
    return OUT


if __name__ == "__main__":
    print(build_library(verbose=True, ptxas_info="-v" in sys.argv, force="-f" in sys.argv))
