"""The C-ABI library builds, loads without a GPU and exports every function
that include/pepsi.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pepsi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pepsi_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2310_14565_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pepsi_setup", "pepsi_server_load", "pepsi_query", "pepsi_eval", "pepsi_decrypt",
                     "pepsi_destroy", "pepsi_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    for name in declared_functions():
        assert hasattr(built_lib, name), name


def test_binding_covers_every_declared_symbol():
    import paper_2310_14565_gb300 as pepsi

    assert set(declared_functions()) == set(pepsi.SYMBOLS)


def test_strerror_without_gpu(built_lib):
    built_lib.pepsi_strerror.restype = ctypes.c_char_p
    assert built_lib.pepsi_strerror(0) == b"ok"
    assert b"overflow" in built_lib.pepsi_strerror(2)
