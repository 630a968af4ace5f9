"""The C-ABI library builds, loads and exports every entry point declared in
include/bddc.h (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_0910_5863_gb300 import bddc as B
from paper_0910_5863_gb300 import build as BUILD

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"BDDC_API[^;(]*?\b(bddc_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    BUILD.build()
    return ctypes.CDLL(BUILD.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n
    assert set(B.EXPORTS) <= names


def test_host_only_calls(lib):
    B.load()
    opt = B.Options()
    B._lib.bddc_default_options(ctypes.byref(opt))
    assert opt.tol == 1e-8 and opt.maxit == 1000 and opt.precision == B.FP64
    assert opt.dev_alloc is None and opt.dev_free is None and opt.alloc_ctx is None
    assert B._lib.bddc_status_str(3) == b"matrix not positive definite"
    assert B._lib.bddc_launch_count(None) == 0
    assert B._lib.bddc_setup(None) == 1
    assert B._lib.bddc_set_corners(None, 0, None) == 1
    assert B._lib.bddc_select_corners(None, None) == 1
    assert B._lib.bddc_set_problem(None, 1, 1, 1, None, None, 0) == 1
    assert B._lib.bddc_set_edge_rows(None, 1) == 1
    assert B._lib.bddc_get_edge_rows(None, None, None) == 1
