"""Compile the CUDA library (csrc/*.cu) for sm_103a into an in-tree libjd.so.

Every translation unit is compiled in parallel with nvcc, then linked with the static
CUDA runtime.  The result sits next to this file and is what the Python binding loads.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libjd.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# host code: no floating-point contraction, so host arithmetic (thresholds, the unit
# combine) rounds the same on every host architecture
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-ffp-contract=off",
                     "-I", INCLUDE, "-I", CSRC, "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libjd.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
                  + glob.glob(os.path.join(INCLUDE, "*.h")))


def _fingerprint(src: str) -> str:
    h = hashlib.sha1()
    for f in [src] + _headers():
        with open(f, "rb") as fh:
            h.update(fh.read())
    h.update(" ".join(NVCC_FLAGS).encode())
    return h.hexdigest()[:16]


def _compile(src: str, extra=()) -> str:
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + "." + _fingerprint(src) + ".o")
    if os.path.exists(obj):
        return obj
    tmp = obj + f".tmp{os.getpid()}"
    cmd = [nvcc()] + NVCC_FLAGS + list(extra) + ["-c", src, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr[-6000:]}")
    os.replace(tmp, obj)
    return obj


def build(jobs: int | None = None, verbose: bool = False, extra=()) -> str:
    """Build libjd.so (incremental: objects are keyed by source + header hashes)."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = _sources()
    jobs = jobs or max(1, min(len(srcs), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), srcs))
    key = hashlib.sha1("".join(sorted(objs)).encode()).hexdigest()[:16]
    stamp = os.path.join(BUILD, "libjd.stamp")
    if os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read() == key:
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as fh:
        fh.write(key)
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build(verbose=True)
