"""GPU parity of kernel 3, several walkers per sample (LAP_OPT_KERNEL = 3,
LAP_OPT_WALKERS lanes share one Wilson run; Section 3.4, stack
representation and Fig. 1: the popped cycles do not depend on the order in
which the walkers find them).

Integer outputs (visits per node, uniform-walk passes, sum Y1, sum Y2,
per-sample Y1 and Y2) must be bit-exact with the sequential CPU oracle for
every walker count (2, 4, 8, 16 and the automatic choice), launch shape and
graph, including samples the kernel
withdraws (a path longer than a walker's stack) and re-runs with the 8-byte
kernel; FP64 estimates within 1e-12 of the oracle's finalize."""
import numpy as np
import pytest

import oracle
from paper_2311_10290_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2311_10290_gb300.lap import (LAP_OPT_KERNEL, LAP_OPT_PATH_START, LAP_OPT_PATHS,  # noqa: E402
                                        LAP_OPT_SLOTS, LAP_OPT_STACK, LAP_OPT_WALKERS, LAP_STAT_FALLBACKS,
                                        LAP_STAT_KERNEL, LAP_STAT_LAST_KERNEL, LapGraph)


def run3(g, seed, omega, walkers=0, root=-1, slots=None, stack=None, trace=False, start=None, ws=1 << 27,
         splits=None, paths=False):
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=ws)
    try:
        G.set_option(LAP_OPT_KERNEL, 3)
        G.set_option(LAP_OPT_WALKERS, walkers)
        if paths:
            G.set_option(LAP_OPT_PATHS, 1)
        if slots:
            G.set_option(LAP_OPT_SLOTS, slots)
        if stack:
            G.set_option(LAP_OPT_STACK, stack)
        if start is not None:
            G.set_option(LAP_OPT_PATH_START, start)
        v = G.set_root(root)
        assert G.stat(LAP_STAT_KERNEL) == 3
        y = None
        if trace:
            y = G.sample_trace(omega, seed)
        else:
            for part in (splits or [omega]):
                G.sample(part, seed)
        c1, c2, s = G.counts()
        out = dict(v=v, cnt1=c1, cnt2=c2, sums=s, fallbacks=G.stat(LAP_STAT_FALLBACKS),
                   kernel=G.stat(LAP_STAT_LAST_KERNEL))
        if start is None:
            out.update(ld=G.ldiag(), ecc=G.ecc(), kc=G.kemeny())
        if y is not None:
            out["y1"] = y[0].cpu().numpy().astype(np.uint64)
            out["y2"] = y[1].cpu().numpy().astype(np.uint64)
        return out
    finally:
        G.close()


def assert_counts(r, c, omega):
    assert np.array_equal(r["cnt1"], c.cnt1), np.nonzero(r["cnt1"] != c.cnt1)[0][:10]
    assert np.array_equal(r["cnt2"], c.cnt2), np.nonzero(r["cnt2"] != c.cnt2)[0][:10]
    assert int(r["sums"][0]) == omega and int(r["sums"][1]) == c.sum_y1 and int(r["sums"][2]) == c.sum_y2


CASES = [
    ("k4e_v0", I.k4_minus_edge, 0, 3000),
    ("star50", lambda: I.star(50), -1, 1000),
    ("cycle101", lambda: I.cycle(101), 50, 150),
    ("er1000", I.er_1000, -1, 1500),
    ("ba3000", lambda: I.ba(3000, 3, seed=2), -1, 700),
    ("rmat12", lambda: I.rmat(12, 8, seed=3), -1, 400),
    ("er300_sparse", lambda: I.er(300, 0.012, seed=4), -1, 900),
]


@pytest.mark.parametrize("walkers", [2, 4, 8, 16, 0])
@pytest.mark.parametrize("name,maker,root,omega", CASES, ids=[c[0] for c in CASES])
def test_group_kernel_counts_match_oracle(name, maker, root, omega, walkers):
    g = maker()
    r = run3(g, 2718, omega, walkers=walkers, root=root)
    c = oracle.sample(g.row_ptr, g.col, r["v"], 2718, 0, omega, keep_per_sample=False)
    assert_counts(r, c, omega)
    ld, ec, kc = oracle.finalize(g.row_ptr, r["v"], omega, c.cnt1, c.cnt2, c.sum_y1, c.sum_y2)
    np.testing.assert_allclose(r["ecc"], ec, rtol=1e-12, atol=0)
    assert r["kc"] == pytest.approx(kc, rel=1e-12)


@pytest.mark.parametrize("slots", [1, 5, 64])
def test_group_kernel_per_sample_trace_and_slot_reuse(slots):
    """Few groups, many samples: every group runs several samples in its slot
    (cleared at each start); per-sample Y1 and Y2 equal the oracle's."""
    g = I.ba(2000, 4, seed=9)
    omega = 300
    r = run3(g, 77, omega, walkers=4, slots=slots, trace=True)
    c = oracle.sample(g.row_ptr, g.col, r["v"], 77, 0, omega)
    assert_counts(r, c, omega)
    assert np.array_equal(r["y1"], c.y1) and np.array_equal(r["y2"], c.y2)


def test_group_kernel_split_calls_equal_one_call():
    g = I.rmat(11, 6, seed=5)
    a = run3(g, 3, 500, walkers=8)
    b = run3(g, 3, 500, walkers=8, splits=[7, 193, 300])
    assert np.array_equal(a["cnt1"], b["cnt1"]) and np.array_equal(a["cnt2"], b["cnt2"])
    assert np.array_equal(a["sums"], b["sums"])


def test_group_kernel_withdrawn_samples_are_rerun_exactly():
    """A 16-entry stack per walker cannot hold the long loop-erased paths of a
    path graph rooted at one end: those samples are withdrawn (their repeat
    visits subtracted) and re-run with the 8-byte kernel."""
    g = I.path(200)
    r = run3(g, 11, 64, walkers=4, root=0, stack=16)
    assert r["fallbacks"] > 0
    c = oracle.sample(g.row_ptr, g.col, 0, 11, 0, 64, keep_per_sample=False)
    assert_counts(r, c, 64)


@pytest.mark.parametrize("paths", [False, True], ids=["own_draws", "stack_paths"])
def test_group_kernel_fixed_start_rows(paths):
    g = I.er(300, 0.02, seed=2)
    r = run3(g, 4242, 800, walkers=8, start=17, paths=paths)
    c = oracle.sample(g.row_ptr, g.col, r["v"], 4242, 0, 800, keep_per_sample=False, path_start=17, paths=paths)
    assert_counts(r, c, 800)


@pytest.mark.parametrize("walkers", [8, 16])
def test_group_kernel_full_size_rmat22_small_omega(walkers):
    """The R-MAT scale-22 graph (2.4M nodes, a 162,713-degree hub as the
    root): all counts bit-exact for 32 samples, 8 or 16 walkers each."""
    g = I.rmat_22()
    r = run3(g, 5, 32, walkers=walkers, ws=64 << 20 << 4)
    c = oracle.sample_threads(g.row_ptr, g.col, r["v"], 5, 0, 32, 16)
    assert_counts(r, c, 32)
    assert r["fallbacks"] == 0


@pytest.mark.parametrize("walkers", [2, 4, 8, 16])
@pytest.mark.parametrize("name,maker,root,omega", [c for c in CASES if c[0] in ("k4e_v0", "cycle101", "ba3000",
                                                                                  "rmat12", "er300_sparse")],
                         ids=["k4e_v0", "cycle101", "ba3000", "rmat12", "er300_sparse"])
def test_group_kernel_loop_included_paths_match_oracle(name, maker, root, omega, walkers):
    """LAP_OPT_PATHS = 1 on kernel 3: the two absorbed walks take the
    sample's own stacks; counts bit-exact with the oracle's paths mode."""
    g = maker()
    r = run3(g, 4711, omega, walkers=walkers, root=root, paths=True, splits=[omega // 3, omega - omega // 3])
    assert r["kernel"] == 3
    c = oracle.sample(g.row_ptr, g.col, r["v"], 4711, 0, omega, keep_per_sample=False, paths=True)
    assert_counts(r, c, omega)
    ld, ec, kc = oracle.finalize(g.row_ptr, r["v"], omega, c.cnt1, c.cnt2, c.sum_y1, c.sum_y2)
    np.testing.assert_allclose(r["ecc"], ec, rtol=1e-12, atol=0)
    assert r["kc"] == pytest.approx(kc, rel=1e-12)


@pytest.mark.parametrize("walkers", [4, 16])
def test_group_kernel_paths_departure_cap_withdraws_exactly(walkers):
    """On a path graph rooted at one end, loop-included paths leave some nodes
    255 or more times in one sample: those samples are withdrawn (their
    Wilson and path departures subtracted) and re-run with kernel 1."""
    g = I.path(200)
    r = run3(g, 19, 48, walkers=walkers, root=0, paths=True, trace=True)
    assert r["fallbacks"] > 0
    c = oracle.sample(g.row_ptr, g.col, 0, 19, 0, 48, paths=True)
    assert_counts(r, c, 48)
    assert np.array_equal(r["y1"], c.y1) and np.array_equal(r["y2"], c.y2)
