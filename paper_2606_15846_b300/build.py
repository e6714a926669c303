"""Builds libflashnav.so in-tree for sm_103a (nvcc + g++, no JIT cache).

The geometry translation unit is compiled with FMA contraction off and IEEE
division and square root, so its binary32 arithmetic rounds once per
operation; the host runtime is compiled with -ffp-contract=off for the same
reason (its spawnability test must agree with the device footprint test).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libflashnav.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_GEOMETRY = ["nav_step.cu"]
CU_DEFAULT = ["nav_noalloc.cu", "nav_mlp.cu", "nav_fused.cu", "nav_policy.cu", "nav_learn.cu",
              "nav_gather.cu"]
CPP = ["nav_api.cpp"]


def _run(cmd):
    print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)


def _stale(out, srcs):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(HERE, "..", "include", "flashnav.h"))
    objs = []
    common_nv = ["-std=c++17", "-O3", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off",
                 "-I", os.path.join(HERE, "..", "include")]
    if verbose_ptxas:
        common_nv += ["-Xptxas", "-v"]
    for f in CU_GEOMETRY + CU_DEFAULT:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if force or verbose_ptxas or _stale(obj, [src, *headers]):
            fp = ["-fmad=false", "-prec-div=true", "-prec-sqrt=true", "-ftz=false"] \
                if f in CU_GEOMETRY else []
            _run([NVCC, *common_nv, *fp, "-c", src, "-o", obj])
    for f in CPP:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD, f + ".o")
        objs.append(obj)
        if force or _stale(obj, [src, *headers]):
            _run(["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", "-Wall",
                  "-I", os.path.join(CUDA, "include"), "-I", os.path.join(HERE, "..", "include"),
                  "-c", src, "-o", obj])
    if force or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        _run([NVCC, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl",
              "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv)
