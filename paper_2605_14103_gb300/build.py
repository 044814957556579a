"""Builds libzbus.so in-tree with nvcc for sm_103a (parallel, incremental)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libzbus.so")
LIB_CHECKED = os.path.join(HERE, "libzbus_checked.so")

SOURCES = ["api.cu", "setup.cu", "kernels_f64.cu", "mixed.cu", "group.cu", "tune.cu", "serve.cu",
           "noalloc.cu", "phased.cu", "adjoint.cu", "nr.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps_mtime() -> float:
    m = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".cuh", ".h")):
                m = max(m, os.path.getmtime(os.path.join(d, f)))
    return m


def _compile(src: str, dep_m: float, verbose: bool, build_dir: str = BUILD,
             extra=()) -> str:
    s = os.path.join(CSRC, src)
    o = os.path.join(build_dir, src.replace(".cu", ".o"))
    if os.path.exists(o) and os.path.getmtime(o) >= max(os.path.getmtime(s), dep_m):
        return o
    cmd = [_nvcc(), *ARCH, *FLAGS, *extra, "-c", s, "-o", o]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        print(r.stderr)
    return o


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile every CUDA source and link libzbus.so; returns its path.

    checked=True builds libzbus_checked.so instead (-DZBUS_CHECKED: every
    table-derived index tested before use, see zbus_checked_status)."""
    build_dir = BUILD + "_checked" if checked else BUILD
    lib = LIB_CHECKED if checked else LIB
    extra = ["-DZBUS_CHECKED"] if checked else []
    os.makedirs(build_dir, exist_ok=True)
    dep_m = _deps_mtime()
    if force:
        for f in os.listdir(build_dir):
            if f.endswith(".o"):
                os.remove(os.path.join(build_dir, f))
    with cf.ThreadPoolExecutor(max_workers=min(8, len(SOURCES))) as ex:
        objs = list(ex.map(lambda s: _compile(s, dep_m, verbose, build_dir, extra), SOURCES))
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < newest:
        tmp = lib + ".tmp"
        cmd = [_nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
