"""CPU oracle for the LEWalk hot path (arXiv 2311.10290).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The GPU library never loads it, and it never loads the GPU library.

``lewalk_oracle.c`` is the sampler and finalize (plain single-threaded C,
built with gcc into ``liboracle.so``); ``dense.py`` is the FP64 dense estimand.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lewalk_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile lewalk_oracle.c with gcc (portable flags: no -march)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            p = ctypes.c_void_p
            lib.oracle_sample.restype = ctypes.c_int
            lib.oracle_sample.argtypes = [ctypes.c_int32, p, p, ctypes.c_int32, ctypes.c_uint64,
                                          ctypes.c_uint64, ctypes.c_uint64, p, ctypes.c_int32,
                                          p, p, p, p, p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int32]
            lib.oracle_cyclepop.restype = ctypes.c_int
            lib.oracle_cyclepop.argtypes = [ctypes.c_int32, p, p, ctypes.c_int32, ctypes.c_uint64,
                                            ctypes.c_uint64, ctypes.c_uint64, p, p, p]
            lib.oracle_finalize.restype = None
            lib.oracle_finalize.argtypes = [ctypes.c_int32, p, ctypes.c_int32, ctypes.c_uint64,
                                            p, p, ctypes.c_uint64, ctypes.c_uint64, p, p, p]
            lib.oracle_sample_cv.restype = ctypes.c_int
            lib.oracle_sample_cv.argtypes = [ctypes.c_int32, p, p, ctypes.c_int32, ctypes.c_uint64,
                                             ctypes.c_uint64, ctypes.c_uint64, p, p, p, p, p, p, p, p, p, p,
                                             ctypes.c_int]
            lib.oracle_hitting_walks.restype = ctypes.c_int
            lib.oracle_hitting_walks.argtypes = [ctypes.c_int32, p, p, ctypes.c_int32, ctypes.c_uint64,
                                                 ctypes.c_uint32, p, ctypes.c_uint64]
            lib.oracle_philox_block.restype = None
            lib.oracle_philox_block.argtypes = [p, p, p]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox_block(ctr, key):
    """Philox4x32-10 block for counter words ctr[4] and key words key[2]."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().oracle_philox_block(_ptr(c), _ptr(k), _ptr(out))
    return out


class Counts:
    """Integer state the estimators are built from (all sums over sample ids)."""

    def __init__(self, n):
        self.cnt1 = np.zeros(n, dtype=np.uint64)
        self.cnt2 = np.zeros(n, dtype=np.uint64)
        self.y1 = None      # per-sample Y1 (uint64) when requested
        self.y2 = None
        self.tree = None
        self.sum_y1 = 0
        self.sum_y2 = 0
        self.omega = 0


def sample(row_ptr, col, v, seed, first, count, order=None, keep_per_sample=True,
           keep_tree=False, max_steps=0, paths=False, path_start=-1):
    """Run sample ids [first, first+count) on one thread; returns Counts.
    paths=True: the two absorbed walks are the sample's loop-included paths
    (see oracle_one_sample in lewalk_oracle.c).  path_start >= 0: the first
    absorbed walk (or path) starts at that node instead of a uniform draw, so
    cnt2 / (count d_u) estimates row path_start of L_v^{-1}."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    n = rp.size - 1
    out = Counts(n)
    y1 = np.zeros(count, dtype=np.uint64)
    y2 = np.zeros(count, dtype=np.uint64)
    tree = np.zeros(count * n, dtype=np.int32) if keep_tree else None
    od = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    rc = _load().oracle_sample(n, _ptr(rp), _ptr(cl), int(v), int(seed), int(first), int(count),
                               _ptr(od), 0 if od is None else od.size,
                               _ptr(out.cnt1), _ptr(out.cnt2), _ptr(y1), _ptr(y2), _ptr(tree),
                               int(max_steps), int(bool(paths)), int(path_start))
    if rc != 0:
        raise RuntimeError("oracle_sample failed with code %d" % rc)
    out.sum_y1 = int(y1.sum(dtype=np.uint64))
    out.sum_y2 = int(y2.sum(dtype=np.uint64))
    out.omega = count
    if keep_per_sample:
        out.y1, out.y2 = y1, y2
    if keep_tree:
        out.tree = tree.reshape(count, n)
    return out


def sample_cv(row_ptr, col, v, seed, first, count, h1=None, h2=None, paths=False):
    """oracle.sample plus the control-variate sums: returns (Counts, a1, a2, p2,
    m2 per sample).  h1, h2: int64 potentials (or None)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    n = rp.size - 1
    out = Counts(n)
    y1 = np.zeros(count, dtype=np.uint64)
    y2 = np.zeros(count, dtype=np.uint64)
    m2 = np.zeros(count, dtype=np.float64)
    a1 = np.zeros(n, dtype=np.int64)
    a2 = np.zeros(n, dtype=np.int64)
    p2 = np.zeros(n, dtype=np.int64)
    H1 = None if h1 is None else np.ascontiguousarray(h1, dtype=np.int64)
    H2 = None if h2 is None else np.ascontiguousarray(h2, dtype=np.int64)
    rc = _load().oracle_sample_cv(n, _ptr(rp), _ptr(cl), int(v), int(seed), int(first), int(count),
                                  _ptr(out.cnt1), _ptr(out.cnt2), _ptr(y1), _ptr(y2), _ptr(H1), _ptr(H2),
                                  _ptr(a1), _ptr(a2), _ptr(p2), _ptr(m2), int(bool(paths)))
    if rc != 0:
        raise RuntimeError("oracle_sample_cv failed with code %d" % rc)
    out.y1, out.y2 = y1, y2
    out.sum_y1 = int(y1.sum(dtype=np.uint64))
    out.sum_y2 = int(y2.sum(dtype=np.uint64))
    out.omega = count
    return out, a1, a2, p2, m2


def hitting_walks(row_ptr, col, v, seed, reps, max_steps=0):
    """Per-node sums of `reps` v-absorbed walk lengths from every node (uint64)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    sums = np.zeros(rp.size - 1, dtype=np.uint64)
    rc = _load().oracle_hitting_walks(rp.size - 1, _ptr(rp), _ptr(cl), int(v), int(seed), int(reps),
                                      _ptr(sums), int(max_steps))
    if rc != 0:
        raise RuntimeError("oracle_hitting_walks failed with code %d" % rc)
    return sums


def sample_threads(row_ptr, col, v, seed, first, count, threads, paths=False, path_start=-1):
    """Same counts as sample(), with the sample ids split into `threads`
    contiguous ranges run concurrently (ctypes releases the GIL)."""
    threads = max(1, min(int(threads), int(count))) if count else 1
    bounds = [first + (count * t) // threads for t in range(threads + 1)]

    def run(t):
        return sample(row_ptr, col, v, seed, bounds[t], bounds[t + 1] - bounds[t], keep_per_sample=False,
                      paths=paths, path_start=path_start)

    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(run, range(threads)))
    n = np.asarray(row_ptr).size - 1
    out = Counts(n)
    for p in parts:
        out.cnt1 += p.cnt1
        out.cnt2 += p.cnt2
        out.sum_y1 += p.sum_y1
        out.sum_y2 += p.sum_y2
    out.omega = count
    return out


def cyclepop(row_ptr, col, v, seed, first, count, keep_tree=False):
    """Order-free cycle popping: returns (cnt1, y1 per sample, tree or None)."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    cl = np.ascontiguousarray(col, dtype=np.int32)
    n = rp.size - 1
    cnt1 = np.zeros(n, dtype=np.uint64)
    y1 = np.zeros(count, dtype=np.uint64)
    tree = np.zeros(count * n, dtype=np.int32) if keep_tree else None
    rc = _load().oracle_cyclepop(n, _ptr(rp), _ptr(cl), int(v), int(seed), int(first), int(count),
                                 _ptr(cnt1), _ptr(y1), _ptr(tree))
    if rc != 0:
        raise RuntimeError("oracle_cyclepop failed with code %d" % rc)
    return cnt1, y1, (tree.reshape(count, n) if keep_tree else None)


def finalize(row_ptr, v, omega, cnt1, cnt2, sum_y1, sum_y2):
    """Returns (ldiag[n], ecc[n], kemeny) from the integer counts."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    n = rp.size - 1
    c1 = np.ascontiguousarray(cnt1, dtype=np.uint64)
    c2 = np.ascontiguousarray(cnt2, dtype=np.uint64)
    ld = np.zeros(n)
    ec = np.zeros(n)
    kc = np.zeros(1)
    _load().oracle_finalize(n, _ptr(rp), int(v), int(omega), _ptr(c1), _ptr(c2),
                            int(sum_y1), int(sum_y2), _ptr(ld), _ptr(ec), _ptr(kc))
    return ld, ec, float(kc[0])


def root_max_degree(row_ptr):
    """Landmark v = a highest-degree node, smallest id on ties (Section 6, Parameters)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    d = rp[1:] - rp[:-1]
    return int(np.argmax(d))          # argmax returns the first maximum
