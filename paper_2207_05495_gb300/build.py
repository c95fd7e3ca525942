"""Builds the CUDA library libsw.so in-tree with nvcc, for sm_103a only.

The translation units compile in parallel (one nvcc process each) and are
then linked into one shared library."""

from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
SOURCES = [os.path.join(CSRC, "sw_engine.cu"), os.path.join(CSRC, "sw_beam.cu"), os.path.join(CSRC, "sw_probe.cu")]
DEPS = SOURCES + [os.path.join(CSRC, "sw_kernels.cuh"), os.path.join(CSRC, "sw_internal.h"),
                  os.path.join(ROOT, "include", "sw.h")]
LIB = os.path.join(HERE, "libsw.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return LIB
    tag = f".tmp{os.getpid()}"
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(HERE, os.path.basename(src)[:-3] + tag + ".o")
        cmd = [nvcc(), "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I",
               os.path.join(ROOT, "include"), "-c", "-o", obj, src]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        objs.append(obj)
        procs.append(subprocess.Popen(cmd))
    rcs = [p.wait() for p in procs]
    try:
        if any(rcs):
            raise subprocess.CalledProcessError(max(rcs), "nvcc")
        tmp = LIB + tag
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp] + objs)
        os.replace(tmp, LIB)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
