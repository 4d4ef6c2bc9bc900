"""Build libsmoe.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into one shared
library with the CUDA runtime linked statically (no torch, no Python in the
library).  Called by ``__graft_entry__.build()``; safe to call repeatedly (it
rebuilds only when a source is newer than the library).
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libsmoe.so")
BUILD_DIR = os.path.join(HERE, "_build")
SOURCES = ["bin.cu", "render.cu", "adam.cu", "api.cu", "static_render.cu", "resample.cu",
           "reorder.cu"]
# Issue-rate micro-benchmark (the ALU roofline's per-clock peaks), its own library.
RATES_SRC = "issue_rates.cu"
RATES_LIB = os.path.join(HERE, "libsmoe_rates.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I", INCLUDE]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsmoe.so")
    return path


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "smoe.h"))
    return files


def needs_build() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(RATES_LIB):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(RATES_LIB))
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    def rates_lib():
        tmp = RATES_LIB + ".tmp%d" % os.getpid()
        cmd = [cc, *ARCH, *FLAGS, *extra, "-shared", os.path.join(CSRC, RATES_SRC), "-o", tmp,
               "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {RATES_SRC}:\n{r.stderr}")
        os.replace(tmp, RATES_LIB)

    with ThreadPoolExecutor(max_workers=len(SOURCES) + 1) as ex:
        rates = ex.submit(rates_lib)
        objs = list(ex.map(compile_one, SOURCES))
        rates.result()
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="-f" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "-v" in sys.argv else []))
