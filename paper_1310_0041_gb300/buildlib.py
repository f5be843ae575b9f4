"""Build libgd.so (the solver's C-ABI library) in-tree for sm_103a.

    python -m paper_1310_0041_gb300.buildlib

Compiles the CUDA/C++ translation units in parallel with nvcc
(``-gencode arch=compute_103a,code=sm_103a -lineinfo``) and links them into
``paper_1310_0041_gb300/libgd.so`` with the CUDA runtime linked statically.
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
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgd.so")
SOURCES = ["gd_kernels.cu", "gd_zmarch.cu", "gd_host.cu", "gd_batch.cu", "gd_hybrid.cu", "gd_learn.cu",
           "gd_eig.cpp"]
# sources compiled in parts (-D<macro>=0 .. n-1), one object each, so that a
# unit holding many kernel instantiations compiles on several cores
PARTS = {"gd_zmarch.cu": ("GD_ZMARCH_PART", 5)}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgd.so")


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers += [os.path.join(INCLUDE, h) for h in os.listdir(INCLUDE) if h.endswith(".h")]
    cc = nvcc()
    common = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O3",
              "-I", INCLUDE, "-I", CSRC, *extra_flags]
    jobs = []
    objs = []
    units = []
    for src in SOURCES:
        if src in PARTS:
            macro, n = PARTS[src]
            units += [(src, "%s.p%d.o" % (src, k), ["-D%s=%d" % (macro, k)]) for k in range(n)]
        else:
            units.append((src, src + ".o", []))
    for src, oname, defs in units:
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, oname)
        objs.append(obj)
        if force or _stale(obj, [path, *headers]):
            cmd = [cc, *common, *defs, "-c", path, "-o", obj]
            if src.endswith(".cpp"):
                cmd[1:1] = ["-x", "c++"]
            jobs.append(cmd)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError("compile failed:\n%s\n%s%s" % (" ".join(cmd), p.stdout, p.stderr))
        return p.stderr

    with ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        for msg in ex.map(run, jobs):
            if verbose and msg:
                print(msg)
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        run([cc, "-shared", *ARCH, "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
