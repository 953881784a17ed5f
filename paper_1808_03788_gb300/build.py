"""In-tree build of libaderdg.so (CUDA, sm_103a) with nvcc.

Each translation unit under csrc/ is compiled in parallel, then linked
into paper_1808_03788_gb300/_build/libaderdg.so.  Rebuilds only when a
source is newer than the library.  Run as `python -m paper_1808_03788_gb300.build`.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import re
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libaderdg.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                  "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]
CXXFLAGS = ["-O2", "-fPIC", "-std=c++17", "-ffp-contract=off", "-I", INCLUDE, "-I", CSRC]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libaderdg.so")


INST_SRC = os.path.join(CSRC, "inst.cu")
_PDE_TYPE = {"advection": "Advection<%d>", "euler": "Euler<%d>", "elastic": "Elastic3",
             "diffuse": "DiffuseElastic<%d>"}


def instances():
    """(accessor name, PDE type, d, N, T) of every kernel instance: the
    entries of csrc/instances.h, each in double and float."""
    with open(os.path.join(CSRC, "instances.h")) as f:
        text = f.read()
    out = []
    for tag, d, n in re.findall(r"X\((\w+), (\d), (\d)\)", text):
        pde = _PDE_TYPE[tag] % int(d) if "%d" in _PDE_TYPE[tag] else _PDE_TYPE[tag]
        for t, suffix in (("double", "f64"), ("float", "f32")):
            out.append(("ks_%s%sd_n%s_%s" % (tag, d, n, suffix), pde, int(d), int(n), t))
    if not out:
        raise RuntimeError("no kernel instances found in csrc/instances.h")
    return out


def sources():
    """Translation units other than the instance template inst.cu."""
    srcs = glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp"))
    return sorted(s for s in srcs if s != INST_SRC)


def _deps():
    return sources() + [INST_SRC] + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(INCLUDE, "aderdg.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def _compile(src, extra: list[str]) -> str:
    if isinstance(src, tuple):  # a kernel instance of inst.cu
        name, pde, d, n, t = src
        obj = os.path.join(BUILD, name + ".o")
        defs = ["-DADERDG_INST_NAME=" + name, "-DADERDG_INST_PDE=" + pde, "-DADERDG_INST_DIM=%d" % d,
                "-DADERDG_INST_N=%d" % n, "-DADERDG_INST_T=" + t]
        cmd = [_nvcc(), "-c", INST_SRC, "-o", obj] + NVFLAGS + defs + extra
    elif src.endswith(".cu"):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [_nvcc(), "-c", src, "-o", obj] + NVFLAGS + extra
    else:
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = ["g++", "-c", src, "-o", obj] + CXXFLAGS + [f"-I{os.path.dirname(_nvcc())}/../include"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
    return obj


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile every CUDA/C++ source for sm_103a and link libaderdg.so."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = extra or []
    # the slowest units first: the instances with the most nodes
    srcs = sorted(instances(), key=lambda i: -(i[3] + 1) ** i[2]) + sources()
    workers = min(len(srcs), max(2, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), srcs))
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = [_nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else None)
