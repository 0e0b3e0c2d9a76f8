"""The C-ABI library loads and exports every entry point include/*.h declares.

CPU only: nothing here launches a kernel.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(mf_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libmf():
    from paper_2111_03541_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for core in ("mf_mesh_create", "mf_pattern_build", "mf_assemble", "mf_solve"):
        assert core in names


def test_every_declared_symbol_is_exported(libmf):
    missing = [n for n in declared_symbols() if not hasattr(libmf, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    import paper_2111_03541_gb300 as mf
    assert set(declared_symbols()) <= set(mf.exported_symbols())


def test_last_error_callable_without_gpu(libmf):
    libmf.mf_last_error.restype = ctypes.c_char_p
    assert libmf.mf_last_error() == b""


def test_invalid_arguments_rejected_before_any_launch(libmf):
    # NULL descriptors are refused on the host; no device is touched
    libmf.mf_mesh_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    out = ctypes.c_void_p()
    assert libmf.mf_mesh_create(None, None, ctypes.byref(out)) == 1
    libmf.mf_solve.argtypes = [ctypes.c_void_p] * 6
    assert libmf.mf_solve(None, None, None, None, None, None) == 1
