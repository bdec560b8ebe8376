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


def test_probe_library_is_separate_from_the_method_library(lib):
    """The benchmark's random-access probe is a measurement aid: it is built
    into liblap_probe.so with its own header, and the method's library and
    headers do not carry it."""
    from paper_2311_10290_gb300 import probe
    assert "lap_probe_random_rw" not in declared_functions()
    assert not hasattr(lib, "lap_probe_random_rw")
    assert hasattr(ctypes.CDLL(probe.LIB_PATH), "lap_probe_random_rw")


def test_static_sampler_rejects_sample_ids_beyond_32_bits_on_the_host(lib):
    """lap_sample_static checks its id range before any CUDA call, without
    wrap-around: the ids [first_id, first_id + n_samples) must lie below 2^32.
    (The pointers are never dereferenced on these paths.)"""
    f = lib.lap_sample_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64,
                  ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_void_p]
    fake = ctypes.c_void_p(4096)
    too_large = 6
    for first, count in [(1 << 32, 1), (1, 1 << 32), ((1 << 32) - 1, 2), ((1 << 64) - 1, 2), (0, (1 << 32) + 1),
                         ((1 << 64) - 5, 10)]:
        assert f(10, fake, fake, 0, 1, first, count, fake, fake, fake, None) == too_large, (first, count)
    assert f(10, fake, fake, 0, 1, 0, 0, fake, fake, fake, None) == 1       # no samples
    assert f(1, fake, fake, 0, 1, 0, 1, fake, fake, fake, None) == 1        # n < 2
    lib.lap_static_last_error.restype = ctypes.c_char_p
    f(10, fake, fake, 0, 1, (1 << 32) - 1, 2, fake, fake, fake, None)
    assert b"2^32" in lib.lap_static_last_error()
