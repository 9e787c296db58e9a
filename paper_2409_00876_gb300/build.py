"""Compile libpgsgd.so for sm_103a (GB300) in-tree with nvcc.

The library is plain CUDA C++ with a C ABI; no torch headers are involved, so
it builds without a GPU (nvcc cross-compiles) and loads from any process.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libpgsgd.so")
SOURCES = ["pgsgd_kernels.cu", "pgsgd_api.cu", "pgsgd_noalloc.cu", "pgsgd_grad.cu", "pgsgd_full.cu",
           "pgsgd_batch.cu", "pgsgd_probe.cu"]
HEADERS = ["pgsgd_device.cuh", "pgsgd_internal.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
              "-I", os.path.join(ROOT, "include")]
_lock = threading.Lock()


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpgsgd")


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    files.append(os.path.join(ROOT, "include", "pgsgd.h"))
    files.append(os.path.join(ROOT, "include", "pgsgd_batch.h"))
    files.append(os.path.abspath(__file__))
    return files


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Build (if stale) and return the path of libpgsgd.so."""
    with _lock:
        if not force and not _stale():
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        cc = nvcc()
        procs = []
        objs = []
        for src in SOURCES:
            obj = os.path.join(BUILD, src.replace(".cu", ".o"))
            objs.append(obj)
            cmd = [cc, *ARCH, *NVCC_FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
            if verbose:
                print(" ".join(cmd))
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                                                text=True)))
        for cmd, p in procs:
            out, _ = p.communicate()
            if p.returncode != 0:
                raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{out}")
            if verbose and out:
                print(out)
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stdout}{r.stderr}")
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
