"""Build libdgx.so (the C-ABI CUDA library) in-tree for sm_103a.

Each translation unit in csrc/ is compiled by its own nvcc process, all in
parallel, then linked with ``nvcc -shared``.  Objects go to ``_build/``; the
library lands next to this file as ``libdgx.so``.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libdgx.so")
PEAK_SRC = os.path.join(CSRC, "peak", "fma_peak.cu")
PEAK_LIB = os.path.join(HERE, "libdgxpeak.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    headers = sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
                     glob.glob(os.path.join(ROOT, "include", "*.h")) + [os.path.abspath(__file__)])
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in sources:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            # the FP32-bulk kernels use the fast single-precision division and square root
            # (2 ulp, denormals flushed); FP64 arithmetic is unaffected by these flags
            extra = ["--use_fast_math"] if src.endswith("_f32.cu") else []
            cmd = [nvcc] + ARCH + FLAGS + extra + (["-Xptxas", "-v"] if ptxas_info else []) + ["-c", src, "-o", obj]
            log = open(obj + ".log", "w")
            procs.append((subprocess.Popen(cmd, stdout=log, stderr=subprocess.STDOUT), obj, log))
    failed = []
    for p, obj, log in procs:
        rc = p.wait()
        log.close()
        if rc != 0:
            failed.append(obj)
        if verbose or rc != 0:
            sys.stderr.write(open(obj + ".log").read())
    if failed:
        raise RuntimeError("nvcc failed for: " + ", ".join(os.path.basename(f) for f in failed))
    if force or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"], check=True)
        os.replace(tmp, LIB)
    if force or _stale(PEAK_LIB, [PEAK_SRC]):
        # the arithmetic-peak probe the benchmark reports against (not part of the solver's ABI)
        tmp = PEAK_LIB + f".tmp{os.getpid()}"
        subprocess.run([nvcc] + ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-o", tmp, PEAK_SRC],
                       check=True)
        os.replace(tmp, PEAK_LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
