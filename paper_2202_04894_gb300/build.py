"""Builds libdefmm.so in-tree for sm_103a (nvcc + g++, no cmake).

Translation units are compiled in parallel into ``_build/`` next to this
file and linked into ``libdefmm.so`` in the package directory.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdefmm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                     "-I" + INCLUDE]
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-I" + INCLUDE]

SOURCES = [
    ("plan.cpp", "g++"),
    ("persist.cpp", "g++"),
    ("kernels.cu", "nvcc"),
    ("plan_gpu.cu", "nvcc"),
    ("capi.cu", "nvcc"),
    ("noalloc.cu", "nvcc"),
    ("serve.cu", "nvcc"),
    ("tune.cu", "nvcc"),
    ("gmres.cu", "nvcc"),
]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    raise RuntimeError("nvcc not found")


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compiles every translation unit and links ``libdefmm.so``; returns its path.

    checked=True builds ``libdefmm_checked.so`` instead (objects in their own
    folder): every CUDA unit compiled with DEFMM_CHECKED, so the kernels test
    the table indices they follow and raise the plan's error flag (value 2) on
    one out of range instead of reading outside a table."""
    lib = LIB if not checked else os.path.join(HERE, "libdefmm_checked.so")
    bdir = BUILD if not checked else BUILD + "_checked"
    extra = [] if not checked else ["-DDEFMM_CHECKED"]
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()
    procs, objs = [], []
    for src, tool in SOURCES:
        obj = os.path.join(bdir, src.rsplit(".", 1)[0] + ".o")
        path = os.path.join(CSRC, src)
        if tool == "nvcc":
            cmd = [nvcc] + NVCC_FLAGS + extra + ["-c", path, "-o", obj]
        else:
            cmd = ["g++"] + CXX_FLAGS + ["-c", path, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    for cmd, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s" % (" ".join(cmd), out.decode(errors="replace")))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread", "-ldl"]
    out = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if out.returncode != 0:
        raise RuntimeError("link failed: %s\n%s" % (" ".join(cmd), out.stdout.decode(errors="replace")))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
