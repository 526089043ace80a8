"""Builds libnf.so in-tree with nvcc for sm_103a (GB300).

The translation units are compiled in parallel and linked into
``paper_2110_11392_gb300/libnf.so`` (static CUDA runtime, C ABI only).  The
build is skipped when the library is newer than every source.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from typing import List

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libnf.so")
SOURCES = ["nf_bin.cu", "nf_force.cu", "nf_step.cu", "nf_multipole.cu", "nf_far.cu", "nf_api.cu"]
# the benchmark's multiply-add probe: a library of its own, not part of libnf
PROBE_SRC = os.path.join(CSRC, "probe", "fma_probe.cu")
PROBE_LIB = os.path.join(PKG, "libnf_probe.so")
HEADERS = ["nf_internal.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
LINK_LIBS: List[str] = []
NVCC_FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnf")


def _inputs() -> List[str]:
    files = [os.path.join(CSRC, s) for s in SOURCES + HEADERS]
    files.append(os.path.join(ROOT, "include", "nf.h"))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build_library(force: bool = False, verbose: bool = False, extra_flags: List[str] = ()) -> str:
    """Compile and link libnf.so; returns its path."""
    if not force and not extra_flags and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [cc, *NVCC_FLAGS, *ARCH, *extra_flags, "-I", os.path.join(ROOT, "include"),
               "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((src, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode:
            print(out.decode(errors="replace"))
        if p.returncode:
            failed.append(src)
    if failed:
        raise RuntimeError(f"nvcc failed on {failed}")
    tmp = LIB + f".{os.getpid()}.tmp"
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(cc)), "lib64")
    rpath = ["-Xlinker", "-rpath", "-Xlinker", cuda_lib] if os.path.isdir(cuda_lib) else []
    subprocess.check_call([cc, "-shared", *ARCH, "-o", tmp, *objs, *LINK_LIBS, *rpath])
    os.replace(tmp, LIB)
    return LIB


def build_probe(force: bool = False) -> str:
    """Compile and link the multiply-add probe library (libnf_probe.so)."""
    if not force and os.path.exists(PROBE_LIB) and os.path.getmtime(PROBE_LIB) >= os.path.getmtime(PROBE_SRC):
        return PROBE_LIB
    cc = nvcc()
    tmp = PROBE_LIB + f".{os.getpid()}.tmp"
    subprocess.check_call([cc, *NVCC_FLAGS, *ARCH, "-shared", "-o", tmp, PROBE_SRC])
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


if __name__ == "__main__":
    import sys
    print(build_library(force="--force" in sys.argv, verbose="-v" in sys.argv))
