"""Build libgpa.so (CUDA kernels + C ABI) and libgpa_gen.so (the generator) in-tree.

nvcc compiles every translation unit for sm_103a in parallel; gcc builds the
generator with -ffp-contract=off so that its floating point is identical on
x86 and Arm hosts.  Objects go to ``_build/`` next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INC = os.path.join(ROOT, "include")
OBJ = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgpa.so")
GENLIB = os.path.join(PKG, "libgpa_gen.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["k_alloc.cu", "k_test.cu", "k_search.cu", "k_serve.cu", "k_noalloc.cu", "k_stage.cu", "k_peak.cu",
              "k_alloc_wide.cu", "k_test_wide.cu", "k_alloc_small.cu", "k_probe.cu"]
CPP_SOURCES = ["host.cpp", "serve.cpp", "probe.cpp"]
C_SOURCES = ["gen.c"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgpa")


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def _included_sources(src):
    """The .cu files `src` includes (the capacity builds re-include a kernel source)."""
    out = []
    with open(src) as fh:
        for line in fh:
            line = line.strip()
            if line.startswith("#include") and line.endswith('.cu"'):
                out.append(os.path.join(CSRC, line.split('"')[1]))
    return out


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INC, "gpa.h"))
    jobs = []
    objs = []
    for f in CU_SOURCES:
        src = os.path.join(CSRC, f)
        if not os.path.exists(src):
            continue
        obj = os.path.join(OBJ, f + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + _included_sources(src) + headers):
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INC, "-I", CSRC,
                   "-c", src, "-o", obj]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    for f in CPP_SOURCES:
        src = os.path.join(CSRC, f)
        obj = os.path.join(OBJ, f + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INC, "-I", CSRC, "-c", src,
                         "-o", obj])
    for f in C_SOURCES:
        src = os.path.join(CSRC, f)
        obj = os.path.join(OBJ, f + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append(["gcc", "-O2", "-std=c11", "-fPIC", "-ffp-contract=off", "-I", INC, "-c", src, "-o", obj])
    outputs = []
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for out in ex.map(_run, jobs):
            outputs.append(out)
    if verbose or ptxas_info:
        for o in outputs:
            if o.strip():
                print(o)
    if force or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        _run([nvcc, "-shared", "-cudart", "static", *ARCH, "-o", tmp, *objs, "-lpthread"])
        os.replace(tmp, LIB)
    gen_obj = os.path.join(OBJ, "gen.c.o")
    if force or _stale(GENLIB, [gen_obj]):
        tmp = GENLIB + f".tmp{os.getpid()}"
        _run(["gcc", "-shared", "-o", tmp, gen_obj, "-lpthread"])
        os.replace(tmp, GENLIB)
    return LIB


def build_gen_only() -> str:
    """The generator alone (no CUDA toolkit needed)."""
    os.makedirs(OBJ, exist_ok=True)
    src = os.path.join(CSRC, "gen.c")
    obj = os.path.join(OBJ, "gen.c.o")
    if _stale(obj, [src, os.path.join(INC, "gpa.h")]):
        _run(["gcc", "-O2", "-std=c11", "-fPIC", "-ffp-contract=off", "-I", INC, "-c", src, "-o", obj])
    if _stale(GENLIB, [obj]):
        tmp = GENLIB + f".tmp{os.getpid()}"
        _run(["gcc", "-shared", "-o", tmp, obj, "-lpthread"])
        os.replace(tmp, GENLIB)
    return GENLIB


if __name__ == "__main__":
    import sys
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
