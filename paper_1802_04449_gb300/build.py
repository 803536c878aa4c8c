"""Build libclv.so (the CUDA library behind include/clv.h) for sm_103a, in-tree."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libclv.so")
SOURCES = ["clv_api.cu", "clv_noalloc.cu", "clv_freezeout.cu", "clv_cooperfrye.cu", "clv_charge.cu", "clv_bulk.cu",
           "clv_measure.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -prec-div/-prec-sqrt=false: approximate FP32 division and square root (FP64 unaffected)
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-prec-div=false", "-prec-sqrt=false",
         "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(ROOT, "include", "clv.h"))
    return files


def build(force: bool = False, verbose: bool = False, lib: str | None = None, defines=()) -> str:
    """Compile libclv.so; ``defines`` are extra -D flags (tuning variants go to ``lib``)."""
    os.makedirs(BUILD, exist_ok=True)
    out = lib or LIB
    if not force and not defines and os.path.exists(out):
        t = os.path.getmtime(out)
        if all(os.path.getmtime(f) <= t for f in _deps()):
            return LIB
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        tag = "" if not defines else "_" + str(abs(hash(tuple(defines))))
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + tag + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *[f"-D{d}" for d in defines], "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, len(SOURCES))) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
