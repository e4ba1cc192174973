"""Build libboys.so in-tree with nvcc for sm_103a (GB300).

Every translation unit under ``csrc/`` is compiled in parallel, then linked
into ``paper_2504_07637_gb300/libboys.so``.  Objects and the ptxas resource
report go to ``paper_2504_07637_gb300/_build/``.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libboys.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libboys.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.inc")) + [
        os.path.join(ROOT, "include", "boys.h")
    ]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _deps())


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile (if needed) and return the path of libboys.so."""
    if not force and not stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    procs = []
    objs = []
    for src in _sources():
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        log = open(obj + ".log", "w")
        cmd = [cc, *ARCH, *NVCC_FLAGS, "-c", src, "-o", obj]
        procs.append((subprocess.Popen(cmd, stdout=log, stderr=subprocess.STDOUT), src, log, obj))
        objs.append(obj)
    failed = []
    for p, src, log, obj in procs:
        p.wait()
        log.close()
        if p.returncode != 0:
            failed.append((src, open(obj + ".log").read()))
    if failed:
        msg = "\n".join(f"--- {s}\n{out[-4000:]}" for s, out in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    with open(os.path.join(BUILD, "ptxas.log"), "w") as fh:
        for obj in objs:
            fh.write(open(obj + ".log").read())
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    build_library(force="--force" in sys.argv, verbose=True)
