"""Build libapbf.so (the C-ABI library of include/apbf.h) in-tree for sm_103a,
and libapbf_debug.so, the same sources with the device-side invariant checks
compiled in (APBF_DEBUG_CHECKS=1).

The translation units of both libraries are compiled in parallel with nvcc,
then each set is linked into a shared library next to this file. The CUDA
runtime is linked statically, so the libraries depend only on the driver.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libapbf.so")
LIB_DEBUG = os.path.join(PKG, "libapbf_debug.so")
BUILD = os.path.join(ROOT, "_build")
VARIANTS = [(LIB, "release", []), (LIB_DEBUG, "debug", ["-DAPBF_DEBUG_CHECKS=1"])]
SOURCES = ["kernels.cu", "apbf_capi.cu", "density_static.cu", "serve.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC,-ffp-contract=off,-fvisibility=hidden",
              "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "apbf.h"), __file__]
    return [f for f in files if os.path.isfile(f)]


def needs_build() -> bool:
    if not all(os.path.exists(lib) for lib, _, _ in VARIANTS):
        return True
    t = min(os.path.getmtime(lib) for lib, _, _ in VARIANTS)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Build both libraries if a source changed; returns the release library's path."""
    if not (force or needs_build()):
        return LIB
    jobs = []
    for lib, name, defs in VARIANTS:
        os.makedirs(os.path.join(BUILD, name), exist_ok=True)
        for src in SOURCES:
            jobs.append((os.path.join(CSRC, src), os.path.join(BUILD, name, os.path.splitext(src)[0] + ".o"), defs))

    def compile_one(job):
        src, obj, defs = job
        cmd = [nvcc(), *NVCC_FLAGS, *defs, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), flush=True)
        subprocess.run(cmd, check=True)

    with ThreadPoolExecutor(len(jobs)) as ex:
        list(ex.map(compile_one, jobs))
    for lib, name, _ in VARIANTS:
        objs = [os.path.join(BUILD, name, os.path.splitext(src)[0] + ".o") for src in SOURCES]
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run([nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp, "-cudart", "static"],
                       check=True)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
