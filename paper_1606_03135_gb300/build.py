"""Build the CUDA library (sm_103a) in-tree: paper_1606_03135_gb300/_build/librbffd.so.

Each translation unit is compiled by its own nvcc process in parallel, then linked as a
shared library with the CUDA runtime linked statically.  No torch headers are involved:
the library's boundary is the plain C ABI of include/rbffd.h.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "librbffd.so")
PROBE_LIB = os.path.join(OUT_DIR, "libfp64probe.so")  # FP64 pipe probe (include/fp64_probe.h)
SOURCES = ["knn.cu", "assemble.cu", "api.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--fmad=true", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librbffd.so")


def _deps():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + \
        [os.path.join(ROOT, "include", f) for f in ("rbffd.h", "fp64_probe.h")]


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.exists(PROBE_LIB) and \
            min(os.path.getmtime(LIB), os.path.getmtime(PROBE_LIB)) >= \
            max(os.path.getmtime(f) for f in _deps()):
        return LIB
    cc = nvcc()
    objs = [os.path.join(OUT_DIR, s.replace(".cu", ".o")) for s in SOURCES]

    def one(src, obj):
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return r.stderr

    probe_obj = os.path.join(OUT_DIR, "fp64_probe.o")
    with cf.ThreadPoolExecutor(len(SOURCES) + 1) as ex:
        logs = list(ex.map(one, SOURCES + ["fp64_probe.cu"], objs + [probe_obj]))
    if verbose:
        for l in logs:
            print(l)
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    tmp = PROBE_LIB + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, probe_obj], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed (probe):\n{r.stderr}")
    os.replace(tmp, PROBE_LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "-v" in sys.argv else []))
