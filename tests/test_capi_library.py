"""Host-side checks of the C ABI boundary (no GPU needed).

The library must build for sm_103a, load, and export every function that
include/thermoamg.h declares; the binding must declare the same set.
"""
import ctypes
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def libpath():
    from paper_1804_10060_gb300 import build
    return build.build()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\([^;]*\)\s*;", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for must in ("fem_assemble_elasticity", "amg_setup", "amg_pcg_solve", "tam_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    src = open(os.path.join(ROOT, "paper_1804_10060_gb300", "thermoamg.py")).read()
    missing = [n for n in declared_functions() if f'"{n}"' not in src]
    assert not missing, missing


def test_error_string_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.tam_last_error.restype = ctypes.c_char_p
    lib.tam_matrix_info.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    # a NULL handle is rejected on the host, before any CUDA call
    assert lib.tam_matrix_info(None, None, None, None) == -1
    assert b"NULL" in lib.tam_last_error()
