"""The C-ABI library builds, loads without a GPU and exports every entry point
declared in include/*.h; argument validation that needs no device works on CPU."""
import ctypes
import glob
import os
import re

import pytest

from paper_1711_06203_b300 import binding as hb
from paper_1711_06203_b300 import build as hbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            if m.group(1) not in ("if", "while", "for", "return", "sizeof", "defined"):
                names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def libs():
    hbuild.build()
    return [hb.lib("default"), hb.lib("exact")]


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("hydro_ctx_create", "hydro_ctx_destroy", "hydro_dt", "hydro_advance_box", "hydro_ctx_check",
                 "hydro_strerror"):
        assert must in names


def test_every_declared_symbol_is_exported(libs):
    for L in libs:
        for name in declared_functions():
            assert hasattr(L, name), name


def test_strerror_and_null_checks_without_gpu(libs):
    L = libs[0]
    assert L.hydro_strerror(0) == b"ok"
    assert L.hydro_strerror(-4).startswith(b"non-physical")
    # NULL arguments are rejected before any CUDA call
    assert L.hydro_ctx_create(None, 0) == hb.HYDRO_EINVAL
    assert L.hydro_advance_box(None, None, None, None, ctypes.c_double(1.0), None, None) == hb.HYDRO_EINVAL
    assert L.hydro_dt(None, None, None, None, None) == hb.HYDRO_EINVAL
    assert L.hydro_ctx_check(None) == hb.HYDRO_EINVAL
