"""Build the CUDA library in-tree for sm_103a.

libhydro.so        — the product library (FP64, multiply-add contraction on)
libhydro_exact.so  — the same sources with contraction off (-fmad=false) and
                     IEEE division and square root (HYDRO_IEEE_DIV_SQRT): every
                     operation rounds separately, so its arithmetic is the
                     scheme's operation order with no fused or refined steps
                     (used by the bitwise parity tests)
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["hydro_api.cu", "hydro_step.cu", "hydro_batch.cu", "hydro_level.cu", "hydro_serve.cu",
           "hydro_noalloc.cu", "hydro_amr.cu", "hydro_mol.cu"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return files + [__file__]


def _stale(target):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in _deps())


def build(force=False, verbose=False):
    os.makedirs(OUT, exist_ok=True)
    variants = {"libhydro.so": [], "libhydro_exact.so": ["-fmad=false", "-DHYDRO_IEEE_DIV_SQRT"]}
    for name, extra in variants.items():
        target = os.path.join(OUT, name)
        if not (force or _stale(target)):
            continue
        cmd = [_nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
               "-I", INCLUDE, "-I", CSRC, *extra, "-o", target]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        cmd += [os.path.join(CSRC, s) for s in SOURCES]
        cmd += ["-lcudart", "-Xcompiler", "-pthread"]
        subprocess.run(cmd, check=True)
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(OUT)
