"""Builds the CUDA library ``_build/libbdd_dbca.so`` for sm_103a (in-tree, no cmake), and its
checked variant ``_build/libbdd_dbca_checked.so``: the same library with the sweep kernels
compiled with -DBDD_CHECKED, whose index checks record BDD_EDEVICE instead of reading or
writing out of bounds (loaded instead of the normal one when BDD_DBCA_CHECKED=1).

Each translation unit is compiled by nvcc in parallel, then linked into the shared libraries.
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
LIB_CHECKED = os.path.join(BUILD, "libbdd_dbca_checked.so")
SOURCES = ["compile.cpp", "order.cpp", "kernels.cu", "adjoint.cu", "api.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    files += [os.path.join(CSRC, "internal.h"), os.path.join(CSRC, "device_common.cuh"),
              os.path.join(INCLUDE, "bdd_dbca.h"),
              os.path.abspath(__file__)]
    return files


CHECKED = "kernels.cu"  # the unit whose index checks -DBDD_CHECKED turns on


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(LIB_CHECKED):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_CHECKED))
    return any(os.path.getmtime(f) > t for f in _inputs())


def _compile(job) -> str:
    src, checked = job
    stem = os.path.splitext(src)[0] + ("_checked" if checked else "")
    obj = os.path.join(BUILD, stem + ".o")
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3",
           "-I", INCLUDE, "-I", CSRC, "-c", os.path.join(CSRC, src), "-o", obj]
    if checked:
        cmd += ["-DBDD_CHECKED"]
    if src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    if src.endswith(".cu"):
        with open(os.path.join(BUILD, f"ptxas_{stem}.txt"), "w") as f:
            f.write(res.stderr)
    return obj


def _link(out: str, objs) -> None:
    tmp = out + f".tmp{os.getpid()}"
    res = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"],
                         capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, out)


def build(force: bool = False) -> str:
    """Compile (if any input changed) both libraries; return the path of the normal one."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    jobs = [(src, False) for src in SOURCES] + [(CHECKED, True)]
    # the longest units first, so the parallel build ends with the short ones
    jobs.sort(key=lambda j: (not j[0].startswith("kernels"), j[0]))
    with cf.ThreadPoolExecutor(len(jobs)) as ex:
        objs = dict(zip(jobs, ex.map(_compile, jobs)))
    normal = [objs[(src, False)] for src in SOURCES]
    checked = [objs[(src, src == CHECKED)] for src in SOURCES]
    _link(LIB, normal)
    _link(LIB_CHECKED, checked)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
