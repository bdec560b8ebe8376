"""Binding of the benchmark's random-access probe (``liblap_probe.so``, see
``lap_probe.h`` beside this file).  The probe is a measurement aid, not a
step of the method; it lives in its own library so the method's library
(``liblap.so``) exports only the method."""
from __future__ import annotations

import ctypes
import os

_DIR = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(os.path.dirname(_DIR), "liblap_probe.so")

_lib = None


class ProbeError(RuntimeError):
    pass


def library():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("liblap_probe.so is not built (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    lib.lap_probe_random_rw.restype = ctypes.c_int
    lib.lap_probe_random_rw.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint64, ctypes.c_void_p]
    _lib = lib
    return lib


def lap_probe_random_rw(buf, blocks, rounds, salt=0, stream=0):
    """Random single-byte read-then-write probe over the uint8 CUDA tensor
    `buf`; blocks * 256 * rounds * 4 pairs, asynchronous on `stream` (a
    cudaStream_t as an integer)."""
    st = library().lap_probe_random_rw(ctypes.c_void_p(buf.data_ptr()), int(buf.numel()), int(blocks), int(rounds),
                                       int(salt), ctypes.c_void_p(int(stream)))
    if st != 0:
        raise ProbeError("lap_probe_random_rw failed with status %d" % st)
