"""CPU checks of the C ABI: the library loads and exports every function
declared in include/*.h (no compute calls: there is no GPU here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(lap_[A-Za-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2311_10290_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["lap_graph_create", "lap_set_root", "lap_sample", "lap_ecc", "lap_kemeny",
                     "lap_graph_destroy", "lap_counts", "lap_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_null_handling(lib):
    assert lib.lap_version() >= 10000
    lib.lap_last_error.restype = ctypes.c_char_p
    lib.lap_last_error.argtypes = [ctypes.c_void_p]
    assert lib.lap_last_error(None)
    # NULL handle arguments are rejected before any CUDA call.
    lib.lap_sample.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64]
    assert lib.lap_sample(None, 1, 1) == 1
    lib.lap_graph_destroy.argtypes = [ctypes.c_void_p]
    assert lib.lap_graph_destroy(None) == 0
    lib.lap_graph_create.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    assert lib.lap_graph_create(1, None, None, 0, None) == 1


def test_python_binding_names_match_c_names():
    from paper_2311_10290_gb300 import lap
    for n in declared_functions():
        assert hasattr(lap, n), n
