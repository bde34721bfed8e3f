"""The C-ABI library builds, loads and exports every entry point of include/vote.h
(no GPU needed: nothing here launches work)."""
import ctypes
import os
import re

import pytest

from paper_2107_11810_gb300 import build, vote

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "vote.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vote_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return vote.load()


def test_header_declares_the_binding_exports():
    assert declared_symbols() == sorted(vote.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_last_error_callable_without_gpu(lib):
    assert isinstance(lib.vote_last_error(), bytes)


def test_create_rejects_bad_shapes_before_touching_the_gpu(lib):
    import numpy as np
    h = ctypes.c_void_p()
    eps = np.array([0.01, 0.01])
    bounds = np.array([-1.0, 1.0, -1.0, 2.0])
    rc = lib.vote_create(1, 3, 1, eps.ctypes.data_as(ctypes.c_void_p), bounds.ctypes.data_as(ctypes.c_void_p),
                         ctypes.byref(h))
    assert rc == 1 and not h.value
    bad = np.array([0.0, 0.01])
    rc = lib.vote_create(1, 2, 1, bad.ctypes.data_as(ctypes.c_void_p), bounds.ctypes.data_as(ctypes.c_void_p),
                         ctypes.byref(h))
    assert rc == 1 and not h.value
    assert b"eps" in lib.vote_last_error()
