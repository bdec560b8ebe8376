"""Seeded synthetic input graphs (shared by the GPU path's tests/benchmarks and
by the CPU oracle's tests).  Holds none of the sampling method's arithmetic.

Every graph is returned as a :class:`Graph` in the CSR form the method assumes
(Section 2 of the paper: unweighted, undirected, connected): int32 ``row_ptr``
and ``col``, each edge in both directions, rows sorted, no self-loops or
duplicates.

Workload recipes (the paper's SNAP graphs are not available; these stand in
for their shape: power-law degrees, small diameter, easy-to-hit hub root):

* ``er_1000``         Erdos-Renyi G(1000, 0.01), seed 0, largest component.
* ``ba_1m``           Barabasi-Albert n = 10^6, m = 5 (about 5M edges), seed 0.
* ``rmat_22``         R-MAT (0.57, 0.19, 0.19, 0.05), scale 22, 16 * 2^22 generated
                      edges, symmetrised, de-duplicated, largest component.
* ``batch_graphs``    the 512 uneven graphs of the batched workload.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lib = None
_lock = threading.Lock()


class _GG(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("arcs", ctypes.c_int64),
                ("row_ptr", ctypes.POINTER(ctypes.c_int32)), ("col", ctypes.POINTER(ctypes.c_int32)),
                ("orig_id", ctypes.POINTER(ctypes.c_int32))]


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            gp = ctypes.POINTER(_GG)
            lib.gg_from_edges.restype = gp
            lib.gg_from_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            lib.gg_er.restype = gp
            lib.gg_er.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_uint64, ctypes.c_int]
            lib.gg_ba.restype = gp
            lib.gg_ba.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64]
            lib.gg_rmat.restype = gp
            lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_int]
            lib.gg_free.restype = None
            lib.gg_free.argtypes = [gp]
            _lib = lib
    return _lib


@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray      # int32[n+1]
    col: np.ndarray          # int32[2m]
    name: str = ""
    orig_id: np.ndarray | None = None

    @property
    def arcs(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def degree(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))


def _take(ptr, name) -> Graph:
    if not ptr:
        raise MemoryError("graph generator failed for " + name)
    g = ptr.contents
    n, arcs = int(g.n), int(g.arcs)
    rp = np.ctypeslib.as_array(g.row_ptr, shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(g.col, shape=(max(arcs, 1),))[:arcs].copy()
    orig = np.ctypeslib.as_array(g.orig_id, shape=(max(n, 1),))[:n].copy()
    _load().gg_free(ptr)
    return Graph(n, rp, col, name, orig)


def from_edges(n, edges, lcc=False, name="edges") -> Graph:
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    s = np.ascontiguousarray(e[:, 0])
    t = np.ascontiguousarray(e[:, 1])
    return _take(_load().gg_from_edges(int(n), int(e.shape[0]), s.ctypes.data, t.ctypes.data, int(lcc)), name)


def er(n, p, seed=0, lcc=True) -> Graph:
    return _take(_load().gg_er(int(n), float(p), int(seed), int(lcc)), "er(%d,%g,seed=%d)" % (n, p, seed))


def ba(n, m, seed=0) -> Graph:
    return _take(_load().gg_ba(int(n), int(m), int(seed)), "ba(%d,%d,seed=%d)" % (n, m, seed))


def rmat(scale, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=0, lcc=True, n_edges=None) -> Graph:
    ne = int(n_edges if n_edges is not None else edge_factor * (1 << scale))
    return _take(_load().gg_rmat(int(scale), ne, float(a), float(b), float(c), int(seed), int(lcc)),
                 "rmat(%d,%s,seed=%d)" % (scale, edge_factor, seed))


# ---------------------------------------------------------------- small graphs

def complete(n) -> Graph:
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], name="K%d" % n)


def path(n) -> Graph:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], name="P%d" % n)


def cycle(n) -> Graph:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], name="C%d" % n)


def star(n) -> Graph:
    """Hub 0 joined to leaves 1..n-1."""
    return from_edges(n, [(0, i) for i in range(1, n)], name="S%d" % n)


def k4_minus_edge() -> Graph:
    """K4 without the edge {0, 3}: nodes 0 and 3 have degree 2, nodes 1, 2 degree 3."""
    return from_edges(4, [(0, 1), (0, 2), (1, 2), (1, 3), (2, 3)], name="K4-e")


# ------------------------------------------------------------------ workloads

def er_1000(seed=0) -> Graph:
    g = er(1000, 0.01, seed=seed, lcc=True)
    g.name = "er_1000_p0.01_lcc"
    return g


def ba_1m(seed=0) -> Graph:
    g = ba(1_000_000, 5, seed=seed)
    g.name = "ba_n1e6_m5"
    return g


def rmat_22(seed=0) -> Graph:
    g = rmat(22, 16, seed=seed)
    g.name = "rmat_s22_ef16_lcc"
    return g


def batch_spec(count=512, n_lo=1_000, n_hi=1_000_000, seed0=0):
    """(family, n, avg_degree, seed) for the uneven batch: family by seed mod 3
    (ER, BA, R-MAT), n log-uniform in [n_lo, n_hi], average degree uniform in
    [4, 32], both drawn from numpy's PCG64 seeded with 1000003 + seed."""
    out = []
    for k in range(count):
        s = seed0 + k
        h = np.random.Generator(np.random.PCG64(1_000_003 + s))
        n = int(round(math.exp(h.uniform(math.log(n_lo), math.log(n_hi)))))
        deg = float(h.uniform(4.0, 32.0))
        out.append((("er", "ba", "rmat")[s % 3], n, deg, s))
    return out


def batch_graph(family, n, deg, seed) -> Graph:
    if family == "er":
        g = er(n, min(1.0, deg / max(n - 1, 1)), seed=seed, lcc=True)
    elif family == "ba":
        g = ba(n, max(1, int(round(deg / 2))), seed=seed)
    else:
        scale = max(4, int(math.ceil(math.log2(n))))
        g = rmat(scale, n_edges=int(round(deg / 2 * n)), seed=seed, lcc=True)
    g.name = "%s(n=%d,deg=%.1f,seed=%d)" % (family, n, deg, seed)
    return g


def batch_graphs(spec, threads=None):
    """batch_graph for every entry of `spec`, generated on `threads` host
    threads (the C generator releases the GIL and keeps no global state)."""
    from concurrent.futures import ThreadPoolExecutor
    threads = threads or max(1, min(len(spec), os.cpu_count() or 4))
    order = sorted(range(len(spec)), key=lambda k: -spec[k][1])      # large graphs first
    out = [None] * len(spec)

    def run(k):
        out[k] = batch_graph(*spec[k])

    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(run, order))
    return out
