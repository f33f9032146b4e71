"""Builds the CUDA library ``_build/libbdd_dbca.so`` for sm_103a (in-tree, no cmake).

Each translation unit is compiled by nvcc in parallel, then linked into one shared library.
ptxas register / spill / shared-memory reports of the device code go to
``_build/ptxas_<unit>.txt``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libbdd_dbca.so")
SOURCES = ["compile.cpp", "order.cpp", "kernels.cu", "adjoint.cu", "api.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, "internal.h"), os.path.join(CSRC, "device_common.cuh"),
              os.path.join(INCLUDE, "bdd_dbca.h"),
              os.path.abspath(__file__)]
    return files


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def _compile(src: str) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
           "-I", INCLUDE, "-I", CSRC, "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    if src.endswith(".cu"):
        with open(os.path.join(BUILD, f"ptxas_{os.path.splitext(src)[0]}.txt"), "w") as f:
            f.write(res.stderr)
    return obj


def build(force: bool = False) -> str:
    """Compile (if any input changed) and return the path of the shared library."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    tmp = LIB + f".tmp{os.getpid()}"
    res = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"],
                         capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
