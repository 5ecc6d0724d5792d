"""Builds libnefe.so in-tree with nvcc for sm_103a (no cmake, no torch extension machinery).

    python -m paper_2103_10449_gb300.build [--force] [--debug]

Each translation unit is compiled in parallel into ``_build/`` and linked into
``paper_2103_10449_gb300/libnefe.so`` (CUDA runtime linked statically).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libnefe.so")
# Debug build: the same sources with NEFE_DEBUG_BOUNDS (index checks on every atom index read
# from device data; a bad index sets NEFE_ERR_CELL instead of being dereferenced).
LIB_DEBUG = os.path.join(PKG, "libnefe_debug.so")
SOURCES = ["nefe_kernels.cu", "nefe_api.cu", "nefe_engine.cu", "nefe_noalloc.cu", "nefe_adjoint.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The adjoint unit is built without FMA contraction, so the real parts of its dual-number
# kernel round exactly like its plain FP64 kernel (identical trajectories in the forward, the
# tangent-linear and the recomputed runs).
EXTRA = {"nefe_adjoint.cu": ["-fmad=false"]}
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnefe")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "nefe.h"))
    return files


def needs_build(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    if not force and not needs_build(debug):
        return lib
    nvcc = _nvcc()
    bdir = BUILD + "_debug" if debug else BUILD
    os.makedirs(bdir, exist_ok=True)
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(bdir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, *ARCH, *FLAGS, *EXTRA.get(src, []), *(["-DNEFE_DEBUG_BOUNDS"] if debug else []),
               "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(f"--- {src}\n{out.decode(errors='replace')}")
        elif verbose and out:
            print(out.decode(errors="replace"))
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", *objs, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
