"""Planted-mistake copies of the CPU oracle (test infrastructure only).

A pin is only worth something if a plausible slip in the oracle fails it.
`planted(tmp_dir, edits)` compiles a copy of the oracle's C++ sources with
each (original, replacement) text edit applied to `ctu_ppm.cpp` -- every
original must occur exactly once, so an edit can never silently miss -- and
returns a context manager under which the `oracle` module's functions run the
altered library instead of the real one.
"""
import contextlib
import os
import shutil
import subprocess

import oracle

ORACLE_DIR = os.path.dirname(os.path.abspath(oracle.__file__))
FILES = ("ctu_ppm.cpp", "exact_riemann.cpp", "oracle.h", "flopcount.h")


def build_planted(tmp_dir, edits):
    os.makedirs(tmp_dir, exist_ok=True)
    for f in FILES:
        shutil.copy(os.path.join(ORACLE_DIR, f), tmp_dir)
    path = os.path.join(tmp_dir, "ctu_ppm.cpp")
    src = open(path).read()
    for old, new in edits:
        assert src.count(old) == 1, f"planted edit does not match the oracle exactly once: {old!r}"
        src = src.replace(old, new)
    with open(path, "w") as f:
        f.write(src)
    out = os.path.join(tmp_dir, "liboracle_planted.so")
    subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                    "-fopenmp", "-I", tmp_dir, "-o", out, path, os.path.join(tmp_dir, "exact_riemann.cpp")],
                   check=True)
    return out


@contextlib.contextmanager
def planted(tmp_dir, edits):
    lib = oracle.load(build_planted(str(tmp_dir), edits))
    real = oracle._lib()
    oracle._libs["liboracle.so"] = lib
    try:
        yield
    finally:
        oracle._libs["liboracle.so"] = real
