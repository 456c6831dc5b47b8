"""Compile the CUDA libraries in-tree for sm_103a (explicit nvcc, no cmake).

libpmplus.so   the hashing library (C ABI: include/pmplus.h)
libpmppeaks.so microbenchmarks for the roofline denominators (bench only)
"""
from __future__ import annotations

import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libpmplus.so")
PEAKS_LIB = os.path.join(PKG, "libpmppeaks.so")
TARGETS = {LIB: ("pmplus.cu", "pm_server.cu"), PEAKS_LIB: ("peaks.cu",)}
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    "-shared", "-Xcompiler", "-fPIC",
]


def sources():
    out = []
    for d in (CSRC, os.path.join(os.path.dirname(PKG), "include")):
        for f in sorted(os.listdir(d)):
            if f.endswith((".cu", ".cuh", ".h")):
                out.append(os.path.join(d, f))
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    """Build every library that is older than its sources (in parallel)."""
    newest = max(map(os.path.getmtime, sources()))
    procs = []
    for lib, srcs in TARGETS.items():
        if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
            continue
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [NVCC] + FLAGS + (["-Xptxas", "-v"] if verbose else []) + [
            "-o", tmp] + [os.path.join(CSRC, src) for src in srcs]
        procs.append((subprocess.Popen(cmd), tmp, lib, cmd))
    for p, tmp, lib, cmd in procs:
        if p.wait() != 0:
            raise subprocess.CalledProcessError(p.returncode, cmd)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
