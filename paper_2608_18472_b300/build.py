"""Build the native library libtdz.so in-tree (nvcc for sm_103a + the host C++ part).

Usage: python paper_2608_18472_b300/build.py [--verbose] [--force]
(run by path: importing the package would load the library being rebuilt)
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libtdz.so")
SOURCES_CU = ["tdz_cn1d.cu", "tdz_nd.cu", "tdz_spectrum.cu", "tdz_eigen.cu", "tdz_probe.cu", "tdz_tc.cu"]
SOURCES_CPP = ["tdz_host.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _newer(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, force: bool = False) -> str:
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "tdz.h")]
    if not force and not _newer(LIB, deps):
        return LIB
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    objs = []
    for src in SOURCES_CPP:
        obj = os.path.join(objdir, src + ".o")
        cmd = ["g++", "-O3", "-std=c++17", "-fPIC", "-Wall", "-I", INCLUDE, "-I", CSRC, "-I", "/usr/local/cuda/include",
               "-c", os.path.join(CSRC, src), "-o", obj]
        _run(cmd, verbose)
        objs.append(obj)
    for src in SOURCES_CU:
        obj = os.path.join(objdir, src + ".o")
        cmd = ["nvcc", *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
               "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        _run(cmd, verbose)
        objs.append(obj)
    cudalib = "/usr/local/cuda/lib64"
    cmd = ["nvcc", *ARCH, "-shared", "-o", LIB, *objs, "-L", cudalib, "-lcudart", "-lcublas", "-lcusolver",
           "-Xlinker", "-rpath", "-Xlinker", cudalib]
    _run(cmd, verbose)
    return LIB


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if verbose or r.returncode != 0:
        sys.stdout.write(r.stdout)
        sys.stdout.write(r.stderr)
    if r.returncode != 0:
        raise RuntimeError(f"build step failed: {' '.join(cmd[:3])} ...")


if __name__ == "__main__":
    build(verbose="--verbose" in sys.argv, force="--force" in sys.argv)
    print(LIB)
