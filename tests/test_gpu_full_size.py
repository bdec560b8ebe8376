"""Parity at the full sizes of the two large workloads, in the launch shapes
the benchmark uses.

* Barabasi-Albert n = 10^6, m = 5: complete counts (every node's visits and
  passes, sum Y1, sum Y2) bit-exact against the oracle with several samples
  per lane (256 lanes, 2048 samples: 8 per lane, so the per-slot epoch bits
  and count-table tags separate consecutive samples of one lane).
* R-MAT scale 22, edge factor 16, largest component (2.4M nodes, 1.28e8
  arcs, a 162,713-degree hub as the root): complete counts bit-exact for 48
  samples on the 8-byte and 1-byte kernels, and the benchmark's own launch
  (16,384 samples, the default workspace: the several-walkers kernel)
  checked on sampled ids one by one plus invariants that hold at any size.

Counts are integers: compared bit for bit."""
import os

import numpy as np
import pytest

import oracle
from paper_2311_10290_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2311_10290_gb300.lap import (LAP_OPT_KERNEL, LAP_OPT_SLOTS, LAP_STAT_FALLBACKS,  # noqa: E402
                                        LAP_STAT_KERNEL, LAP_STAT_LAST_KERNEL, LapGraph)

THREADS = max(1, min(16, os.cpu_count() or 1))


def full_counts(g, seed, omega, kernel=None, slots=None, ws=None):
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=ws)
    try:
        if kernel:
            G.set_option(LAP_OPT_KERNEL, kernel)
        if slots:
            G.set_option(LAP_OPT_SLOTS, slots)
        v = G.set_root()
        G.sample(omega, seed)
        c1, c2, s = G.counts()
        return v, c1, c2, s, G.stat(LAP_STAT_FALLBACKS)
    finally:
        G.close()


def assert_counts(v, c1, c2, s, c, omega):
    assert int(s[0]) == omega
    assert np.array_equal(c1, c.cnt1), np.nonzero(c1 != c.cnt1)[0][:10]
    assert np.array_equal(c2, c.cnt2), np.nonzero(c2 != c.cnt2)[0][:10]
    assert int(s[1]) == c.sum_y1 and int(s[2]) == c.sum_y2


def test_full_size_ba_several_samples_per_lane():
    g = I.ba_1m()
    omega, seed = 2048, 99
    v, c1, c2, s, _ = full_counts(g, seed, omega, kernel=2, slots=256)
    c = oracle.sample_threads(g.row_ptr, g.col, v, seed, 0, omega, THREADS)
    assert_counts(v, c1, c2, s, c, omega)


@pytest.fixture(scope="module")
def rmat22():
    return I.rmat_22()


@pytest.mark.parametrize("kernel", [1, 2], ids=["wide", "compact"])
def test_full_size_rmat22_counts_small_omega(rmat22, kernel):
    g = rmat22
    omega, seed = 48, 5
    v, c1, c2, s, _ = full_counts(g, seed, omega, kernel=kernel, ws=64 * 8 * g.n)
    assert v == int(np.argmax(np.diff(g.row_ptr)))
    c = oracle.sample_threads(g.row_ptr, g.col, v, seed, 0, omega, THREADS)
    assert_counts(v, c1, c2, s, c, omega)


def test_full_size_rmat22_bench_launch_sampled(rmat22):
    """The benchmark's launch on this graph: 16,384 samples with the default
    workspace (the 1-byte kernel, every sample in flight at once)."""
    g = rmat22
    omega, seed = 16384, 2024
    G = LapGraph(g.row_ptr, g.col)
    try:
        v = G.set_root()
        assert G.stat(LAP_STAT_KERNEL) == 2
        y1, y2 = G.sample_trace(omega, seed)
        c1, c2, s = G.counts()
        assert G.stat(LAP_STAT_FALLBACKS) == 0
        assert G.stat(LAP_STAT_LAST_KERNEL) == 3             # several walkers per sample at this size
        y1 = y1.cpu().numpy().astype(np.uint64)
        y2 = y2.cpu().numpy().astype(np.uint64)
    finally:
        G.close()
    assert int(s[0]) == omega and int(s[1]) == int(y1.sum()) and int(s[2]) == int(y2.sum())
    assert int(c1.sum()) == int(s[1])            # every Wilson step is one visit
    mask = np.ones(g.n, bool)
    mask[v] = False
    assert c1[v] == 0 and np.all(c1[mask] >= omega)   # every non-root node joins every tree
    assert c2[v] == 0
    ids = np.unique(np.linspace(0, omega - 1, 12).astype(np.int64))
    for i in ids:
        c = oracle.sample(g.row_ptr, g.col, v, seed, int(i), 1)
        assert c.y1[0] == y1[i] and c.y2[0] == y2[i], i
