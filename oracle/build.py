"""Build the CPU oracle shared libraries (test infrastructure only).

liboracle.so        — the FP64 oracle (OpenMP over zones; -ffp-contract=off,
                      no fast-math, so every multiply and add rounds separately)
liboracle_count.so  — the same source with an operation-counting `real`, used to
                      state the algorithmic FP64 operation count per zone-update
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_build")
SRC = [os.path.join(HERE, "ctu_ppm.cpp"), os.path.join(HERE, "exact_riemann.cpp")]
BASE = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
        "-fno-fast-math", "-I", HERE]


def _newer(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False):
    os.makedirs(OUT, exist_ok=True)
    deps = SRC + [os.path.join(HERE, "oracle.h"), os.path.join(HERE, "flopcount.h"), __file__]
    libs = {
        "liboracle.so": BASE + ["-fopenmp"],
        "liboracle_count.so": BASE + ["-DORACLE_COUNT_FLOPS"],
    }
    for name, flags in libs.items():
        target = os.path.join(OUT, name)
        if force or _newer(target, deps):
            cmd = flags + ["-o", target] + SRC
            subprocess.run(cmd, check=True)
    return OUT


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print(OUT)
