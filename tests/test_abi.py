"""The C-ABI library loads on a machine without a GPU and exports every
symbol that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names.update(re.findall(r"SPGEMM_API\s+[\w\s\*]*?\b(spgemm_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import paper_1804_00695_gb300 as sg
    from paper_1804_00695_gb300 import _build
    _build.build()
    return ctypes.CDLL(sg.LIB_PATH)


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("spgemm_symbolic", "spgemm_numeric", "spgemm_create", "spgemm_destroy"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_version_string(lib):
    lib.spgemm_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.spgemm_version()


def test_binding_configures_every_entry_point():
    import paper_1804_00695_gb300 as sg
    lib = sg.load()
    for name in declared_symbols():
        assert getattr(lib, name).argtypes is not None, f"binding lacks {name}"
