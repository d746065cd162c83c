"""Build the tracker's shared library in-tree with nvcc for sm_103a.

libtpcca.so holds the C ABI of include/tpc_tracker.h.  The floating-point
kernels are compiled twice: -fmad=false (namespace tpc_exact, IEEE division
and square root, bit-exact against an FP32 CPU evaluation) and a production
build (tpc_fast: contraction, approximate division and square root, flush
to zero).  The CUDA
runtime is linked statically so the library has no runtime-path needs.
"""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(BUILD, "libtpcca.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# (source, object, extra flags)
UNITS = [
    ("k_int.cu", "k_int.o", []),
    ("k_fp.cu", "k_fp_exact.o", ["-fmad=false", "-DTPC_FP_NS=tpc_exact"]),
    ("k_fp.cu", "k_fp_fast.o", ["-fmad=true", "-prec-div=false", "-prec-sqrt=false", "-ftz=true",
                                "-DTPC_FP_NS=tpc_fast", "-DTPC_FAST_MATH=1"]),
    ("k_refit.cu", "k_refit_exact.o", ["-fmad=false", "-DTPC_FP_NS=tpc_exact"]),
    ("k_refit.cu", "k_refit_fast.o", ["-fmad=true", "-prec-div=false", "-prec-sqrt=false", "-ftz=true",
                                      "-DTPC_FP_NS=tpc_fast", "-DTPC_FAST_MATH=1"]),
    ("tracker.cu", "tracker.o", []),
    ("serve.cu", "serve.o", []),
    ("noalloc.cu", "noalloc.o", []),
]


def nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "tpc_tracker.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libtpcca.so; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    base = [nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
            "-I" + INCLUDE, "-I" + CSRC]
    units = [u for u in UNITS if os.path.exists(os.path.join(CSRC, u[0]))]

    def compile_one(u):
        src, obj, extra = u
        cmd = base + extra + ["-c", os.path.join(CSRC, src), "-o", os.path.join(BUILD, obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose:
            print(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(units)) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp] + \
          [os.path.join(BUILD, o) for o in objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
