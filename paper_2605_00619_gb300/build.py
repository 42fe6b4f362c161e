"""Builds the C-ABI library ``lib/libafe.so`` in-tree for sm_103a (GB300).

First g++ builds and runs ``gen_sref`` (csrc/gen_sref.cpp with the reference-element code),
which writes ``lib/gen/sref_gen.cuh``: the FP32 predictor's reference-stiffness contractions
with the matrix entries as immediates.  Then nvcc compiles the CUDA translation unit and g++
the host topology and reference-element code, in parallel, and ``nvcc -shared`` links them.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "lib")
LIBPATH = os.path.join(LIBDIR, "libafe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(verbose: bool = False, extra_flags=None) -> str:
    os.makedirs(LIBDIR, exist_ok=True)
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    nvcc = _nvcc()
    gendir = os.path.join(LIBDIR, "gen")
    os.makedirs(gendir, exist_ok=True)
    gen_exe = os.path.join(objdir, "gen_sref")
    _run([os.environ.get("CXX", "g++"), "-O2", "-std=c++17", "-I" + CSRC, os.path.join(CSRC, "gen_sref.cpp"),
          os.path.join(CSRC, "refelem.cpp"), "-o", gen_exe])
    _run([gen_exe, os.path.join(gendir, "sref_gen.cuh")])
    common = ["-O3", "-std=c++17", "-I" + INCLUDE, "-I" + CSRC, "-I" + gendir]
    extra = list(extra_flags or [])
    jobs = []
    for src in ("refelem.cpp", "topology.cpp"):
        obj = os.path.join(objdir, src + ".o")
        jobs.append([os.environ.get("CXX", "g++"), *common, "-fPIC", "-Wall", "-c",
                     os.path.join(CSRC, src), "-o", obj])
    cu_obj = os.path.join(objdir, "afe.cu.o")
    jobs.append([nvcc, *common, *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                 *extra, "-c", os.path.join(CSRC, "afe.cu"), "-o", cu_obj])
    with ThreadPoolExecutor(len(jobs)) as ex:
        outs = list(ex.map(_run, jobs))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    objs = [j[-1] for j in jobs]
    _run([nvcc, "-shared", *ARCH, "-o", LIBPATH, *objs, "-lpthread", "-ldl"])
    return LIBPATH


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
