"""Build the C-ABI library libmetad.so for sm_103a with nvcc (in-tree).

Each .cu file is compiled to an object in parallel, then linked into
``paper_2510_06873_gb300/_lib/libmetad.so`` (CUDA runtime linked
statically, so the library needs only the driver).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_lib")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmetad.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "k_neighbors.cu", "k_cv.cu", "k_bias.cu", "k_fes.cu", "k_gcv.cu", "k_static.cu", "k_peak.cu"]
# The FP64 hill and grid arithmetic (bias and free-energy kernels) and the
# FP64 torsion / nearest-distance CVs are compiled without multiply-add
# contraction: every product and sum rounds on its own, so the single-system
# and batched instantiations give the same bits (the compiler may otherwise
# fuse differently in each) and a squared distance rounds as its plain
# definition.
FILE_FLAGS = {"k_bias.cu": ["-fmad=false"], "k_fes.cu": ["-fmad=false"], "k_gcv.cu": ["-fmad=false"]}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmetad.so")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                   "--expt-relaxed-constexpr"] + list(extra)


def _stale(obj, srcs):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile every .cu file and link libmetad.so; returns its path."""
    extra_flags = list(extra_flags) + os.environ.get("METAD_NVCC_FLAGS", "").split()
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(BUILD_DIR, exist_ok=True)
    cc = nvcc()
    headers = [os.path.join(CSRC, "metad_impl.cuh"), os.path.join(CSRC, "hills.cuh"), os.path.join(INCLUDE, "metad.h")]
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    jobs = []
    objs = []
    for s in srcs:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD_DIR, s.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append([cc, "-c", src, "-o", obj] + _flags(list(extra_flags) + FILE_FLAGS.get(s, [])))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout + r.stderr)
        return r

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        list(ex.map(run, jobs))
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".{os.getpid()}.tmp"
        run([cc, "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
