"""Build libfraclap.so in-tree for sm_103a with nvcc (no CMake).

Translation units are compiled in parallel and linked into
paper_1708_03912_gb300/libfraclap.so; object files go to paper_1708_03912_gb300/_build/.
Run ``python -m paper_1708_03912_gb300.build`` (or call build()).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfraclap.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

SOURCES = ["planner.cpp", "cluster.cpp", "capi.cpp", "tune.cpp", "pool.cpp", "assemble.cu", "far_dw.cu", "hmatrix.cu", "adaptive.cu", "refine.cpp", "symmetry.cpp", "hnear.cpp", "linalg.cu", "noalloc.cu", "batch.cu", "mg.cu", "learned.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libfraclap")
    return cand


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    headers.append(os.path.join(INCLUDE, "fraclap.h"))
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", INCLUDE]
    procs = []
    objs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        if not _stale(obj, [path] + headers + [__file__]):
            continue
        cmd = [nvcc, "-c", path, "-o", obj, "-cudart", "shared"] + common
        if src.endswith(".cu"):
            cmd += ARCH + ["--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]
        if verbose:
            print(" ".join(cmd))
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((src, text))
        elif verbose and text.strip():
            print(text)
    if failed:
        msg = "\n".join(f"--- {s} ---\n{t}" for s, t in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    if _stale(LIB, objs):
        cmd = [nvcc, "-shared", "-o", LIB] + objs + ARCH + ["-cudart", "shared"]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
