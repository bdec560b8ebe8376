"""Parity of the CUDA path (called through the C ABI) with the CPU oracle.

Integer outputs (per-node visit and pass counts, sum Y1, sum Y2, per-sample
Y1/Y2) must be bit-exact; FP64 outputs ((L^+)_uu, ECC, Kemeny) must agree with
the oracle's finalize of the same counts to 1e-12 relative: both sides do the
same IEEE operations per node and differ only in the order of two n-term sums
of positive numbers (a few ulp)."""
import numpy as np
import pytest

import oracle
from paper_2311_10290_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2311_10290_gb300.lap import (LAP_OPT_BLOCK, LAP_OPT_KERNEL, LAP_OPT_PATHS, LAP_OPT_SLOTS,  # noqa: E402
                                        LAP_OPT_STACK, LAP_OPT_STEP_LIMIT, LAP_STAT_FALLBACKS,
                                        LAP_STAT_KERNEL, LapError, LapGraph)

RTOL = 1e-12


def gpu_run(g, seed, omega, root=-1, slots=None, block=None, splits=None, ws=None, device_inputs=False,
            kernel=None, stack=None, stats=None, paths=False):
    if device_inputs:
        G = LapGraph(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda(), workspace_bytes=ws)
    else:
        G = LapGraph(g.row_ptr, g.col, workspace_bytes=ws)
    try:
        if slots:
            G.set_option(LAP_OPT_SLOTS, slots)
        if block:
            G.set_option(LAP_OPT_BLOCK, block)
        if kernel:
            G.set_option(LAP_OPT_KERNEL, kernel)
        if stack:
            G.set_option(LAP_OPT_STACK, stack)
        if paths:
            G.set_option(LAP_OPT_PATHS, 1)
        v = G.set_root(root)
        used = G.stat(LAP_STAT_KERNEL)
        for part in (splits or [omega]):
            G.sample(part, seed)
        c1, c2, s = G.counts()
        out = dict(v=v, cnt1=c1, cnt2=c2, sums=s, ld=G.ldiag(), ecc=G.ecc(), kc=G.kemeny(),
                   kernel=used, fallbacks=G.stat(LAP_STAT_FALLBACKS))
        if stats is not None:
            stats.update(kernel=used, fallbacks=out["fallbacks"])
        return out
    finally:
        G.close()


def oracle_run(g, v, seed, omega, threads=1, paths=False):
    if threads > 1:
        return oracle.sample_threads(g.row_ptr, g.col, v, seed, 0, omega, threads, paths=paths)
    return oracle.sample(g.row_ptr, g.col, v, seed, 0, omega, keep_per_sample=False, paths=paths)


def assert_parity(g, r, c, omega):
    assert np.array_equal(r["cnt1"], c.cnt1), np.nonzero(r["cnt1"] != c.cnt1)[0][:10]
    assert np.array_equal(r["cnt2"], c.cnt2), np.nonzero(r["cnt2"] != c.cnt2)[0][:10]
    assert int(r["sums"][0]) == omega
    assert int(r["sums"][1]) == c.sum_y1
    assert int(r["sums"][2]) == c.sum_y2
    ld, ec, kc = oracle.finalize(g.row_ptr, r["v"], omega, c.cnt1, c.cnt2, c.sum_y1, c.sum_y2)
    np.testing.assert_allclose(r["ld"], ld, rtol=RTOL, atol=0)
    np.testing.assert_allclose(r["ecc"], ec, rtol=RTOL, atol=0)
    assert r["kc"] == pytest.approx(kc, rel=RTOL)


CASES = [
    ("k4e_v0", I.k4_minus_edge, 0, 5000),
    ("k4e_auto", I.k4_minus_edge, -1, 777),
    ("star50", lambda: I.star(50), -1, 3001),
    ("path30_end", lambda: I.path(30), 0, 200),
    ("cycle101", lambda: I.cycle(101), 50, 150),
    ("er1000", I.er_1000, -1, 2000),
    ("er300_sparse", lambda: I.er(300, 0.012, seed=4), -1, 999),
    ("ba20000", lambda: I.ba(20000, 3, seed=2), -1, 300),
    ("rmat12", lambda: I.rmat(12, 8, seed=3), -1, 257),
    ("k2", lambda: I.complete(2), 0, 100),
]


@pytest.mark.parametrize("kernel", [1, 2], ids=["wide", "compact"])
@pytest.mark.parametrize("name,maker,root,omega", CASES, ids=[c[0] for c in CASES])
def test_counts_and_estimates_match_oracle(name, maker, root, omega, kernel):
    g = maker()
    seed = 0x5EED0000 + len(name)
    r = gpu_run(g, seed, omega, root=root, kernel=kernel)
    v = r["v"] if root < 0 else root
    if root < 0:
        assert v == oracle.root_max_degree(g.row_ptr)
    c = oracle_run(g, v, seed, omega, threads=4)
    assert_parity(g, r, c, omega)


def test_default_kernels_do_not_fall_back_on_social_graphs():
    """Large calls take the 1-byte kernel (LAP_STAT_KERNEL), a call of a few
    thousand samples the several-walkers kernel (LAP_STAT_LAST_KERNEL); neither
    withdraws a sample on a Barabasi-Albert graph."""
    from paper_2311_10290_gb300.lap import LAP_STAT_LAST_KERNEL
    g = I.ba(20000, 4, seed=1)
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 30)
    try:
        v = G.set_root()
        assert G.stat(LAP_STAT_KERNEL) == 2 and G.stat(LAP_STAT_LAST_KERNEL) == 0
        G.sample(2000, 5)
        assert G.stat(LAP_STAT_LAST_KERNEL) == 3 and G.stat(LAP_STAT_FALLBACKS) == 0
        c1, c2, s = G.counts()
    finally:
        G.close()
    c = oracle_run(g, v, 5, 2000, threads=4)
    assert np.array_equal(c1, c.cnt1) and np.array_equal(c2, c.cnt2)
    assert int(s[1]) == c.sum_y1 and int(s[2]) == c.sum_y2


PATH_CASES = [
    ("k4e_v0", I.k4_minus_edge, 0, 3000),
    ("star50_leaf", lambda: I.star(50), 7, 500),
    ("path40_end", lambda: I.path(40), 39, 120),
    ("er1000", I.er_1000, -1, 1500),
    ("ba20000", lambda: I.ba(20000, 3, seed=2), -1, 200),
    ("rmat12", lambda: I.rmat(12, 8, seed=3), -1, 257),
]


@pytest.mark.parametrize("kernel", [1, 2], ids=["wide", "compact"])
@pytest.mark.parametrize("name,maker,root,omega", PATH_CASES, ids=[c[0] for c in PATH_CASES])
def test_loop_included_paths_match_oracle(name, maker, root, omega, kernel):
    """LAP_OPT_PATHS = 1: the absorbed walks are the loop-included paths of
    each sample's own stacks; counts bit-exact with the oracle's, split calls
    included."""
    g = maker()
    seed = 0xA11CE + len(name)
    r = gpu_run(g, seed, omega, root=root, kernel=kernel, paths=True, splits=[omega // 3, omega - omega // 3])
    v = r["v"]
    c = oracle_run(g, v, seed, omega, threads=4, paths=True)
    assert_parity(g, r, c, omega)
    if kernel == 2:
        assert r["fallbacks"] == 0 or name == "path40_end"


@pytest.mark.parametrize("paths", [False, True], ids=["own_draws", "stack_paths"])
@pytest.mark.parametrize("slots", [1, 3])
def test_count_table_tags_wrap_within_a_lane(slots, paths):
    """A 50-node star rooted at a leaf: the hub draws ~49 times per sample, so
    every sample keeps counts in the lane's table.  With 1 or 3 lanes each lane
    runs hundreds of samples, so the per-sample tags (one per sample, three
    with the paths) wrap and the table is cleared several times; the counts
    stay the oracle's and nothing falls back."""
    g = I.star(50)
    omega = 700
    r = gpu_run(g, 77, omega, root=7, slots=slots, kernel=2, paths=paths)
    c = oracle_run(g, 7, 77, omega, threads=4, paths=paths)
    assert_parity(g, r, c, omega)
    assert r["fallbacks"] == 0


def test_loop_included_paths_overflow_falls_back_exactly():
    """A 256-node path rooted at an end: the paths' departure counts and the
    saturated Wilson counts together overflow the 256-entry table, so samples
    are withdrawn during their paths (cnt2 and CV sums taken back) and re-run
    with the 8-byte kernel; the totals stay the oracle's."""
    g = I.path(256)
    st = {}
    r = gpu_run(g, 9, 60, root=255, kernel=2, paths=True, stats=st)
    c = oracle_run(g, 255, 9, 60, threads=4, paths=True)
    assert_parity(g, r, c, 60)
    assert st["fallbacks"] >= 1


def test_loop_included_paths_lower_the_variance_on_the_small_workload():
    """ER G(1000, 0.01): with the paths on the Wilson stacks the estimates
    from 4096 samples are closer to the dense values than with own draws
    (mean relative ECC error and Kemeny error, over 4 seeds)."""
    import oracle.dense as D
    g = I.er_1000()
    ec_t = D.ecc(g.n, g.row_ptr, g.col)
    kc_t = D.kemeny(g.n, g.row_ptr, g.col)
    err = {False: [], True: []}
    for paths in (False, True):
        for seed in range(4):
            r = gpu_run(g, 100 + seed, 4096, paths=paths)
            err[paths].append((np.mean(np.abs(r["ecc"] - ec_t) / ec_t), abs(r["kc"] - kc_t) / kc_t))
    a, b = np.array(err[False]), np.array(err[True])
    assert b[:, 0].mean() < 0.8 * a[:, 0].mean(), (a, b)
    assert b[:, 1].mean() < 0.5 * a[:, 1].mean(), (a, b)


@pytest.mark.parametrize("name,maker,root,stack,falls_back", [
    ("path_end_counts_table", lambda: I.path(60), 0, None, False),   # far nodes drawn > 30 times: count table
    ("star_leaf_root_hub_table", lambda: I.star(200), 1, None, False),  # the hub is drawn ~199 times per sample
    ("path_far_root_table_heavy", lambda: I.path(256), 255, None, False),  # ~230 of 256 nodes drawn > 30 times
    ("cycle_long_paths", lambda: I.cycle(301), 0, 16, True),         # loop-erased paths longer than the stack
])
def test_compact_overflow_rolls_back_to_wide_kernel(name, maker, root, stack, falls_back):
    """Draw counts above 30 live in the compact kernel's per-sample count
    table; samples that still do not fit (table full, path longer than the
    stack) are withdrawn and re-run with the 8-byte kernel: results stay
    exact either way."""
    g = maker()
    st = {}
    r = gpu_run(g, 3, 300, root=root, kernel=2, stack=stack, splits=[100, 200], stats=st)
    assert (st["fallbacks"] >= 1) == falls_back, st
    c = oracle_run(g, root, 3, 300, threads=4)
    assert_parity(g, r, c, 300)


def test_split_calls_equal_one_call():
    g = I.er(500, 0.02, seed=9)
    a = gpu_run(g, 11, 200)
    b = gpu_run(g, 11, 200, splits=[37, 1, 100, 62])
    for k in ("cnt1", "cnt2", "sums"):
        assert np.array_equal(a[k], b[k])


@pytest.mark.parametrize("kernel", [1, 2], ids=["wide", "compact"])
@pytest.mark.parametrize("slots,block", [(1, 32), (7, 64), (64, 128), (1000, 256), (None, None)])
def test_launch_shape_does_not_change_counts(slots, block, kernel):
    g = I.ba(3000, 2, seed=5)
    ref = gpu_run(g, 3, 500, kernel=1)
    r = gpu_run(g, 3, 500, slots=slots, block=block, kernel=kernel)
    for k in ("cnt1", "cnt2", "sums"):
        assert np.array_equal(ref[k], r[k])


@pytest.mark.parametrize("kernel", [1, 2], ids=["wide", "compact"])
def test_small_workspace_reuses_slots_across_launches(kernel):
    """A 20 kB workspace (2 slots of the compact kernel, 6 of the wide one),
    many samples and several calls: the epoch bit must keep every sample
    independent of the previous contents of its slot."""
    g = I.er(400, 0.03, seed=1)
    v = oracle.root_max_degree(g.row_ptr)
    r = gpu_run(g, 8, 90, ws=20000, splits=[1, 2, 3, 40, 44], kernel=kernel)
    c = oracle_run(g, v, 8, 90)
    assert_parity(g, r, c, 90)


def test_device_resident_csr():
    g = I.rmat(10, 6, seed=8)
    a = gpu_run(g, 21, 100)
    b = gpu_run(g, 21, 100, device_inputs=True)
    for k in ("cnt1", "cnt2", "sums"):
        assert np.array_equal(a[k], b[k])


def test_per_sample_trace_matches_oracle():
    g = I.ba(5000, 4, seed=3)
    G = LapGraph(g.row_ptr, g.col)
    try:
        v = G.set_root()
        G.sample(17, 99)                      # ids 0..16
        y1, y2 = G.sample_trace(40, 99)       # ids 17..56
        torch.cuda.synchronize()
        c = oracle.sample(g.row_ptr, g.col, v, 99, 17, 40)
        assert np.array_equal(y1.cpu().numpy().astype(np.uint64), c.y1)
        assert np.array_equal(y2.cpu().numpy().astype(np.uint64), c.y2)
    finally:
        G.close()


def test_hops_are_bfs_distances():
    g = I.er(600, 0.01, seed=2)
    G = LapGraph(g.row_ptr, g.col)
    try:
        v = G.set_root()
        h = G.hops()
    finally:
        G.close()
    ref = np.full(g.n, -1)
    ref[v] = 0
    frontier = [v]
    while frontier:
        nxt = []
        for u in frontier:
            for w in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]:
                if ref[w] < 0:
                    ref[w] = ref[u] + 1
                    nxt.append(w)
        frontier = nxt
    assert np.array_equal(h, ref)


# ------------------------------------------------------------- error paths

def _expect(status, fn):
    with pytest.raises(LapError) as e:
        fn()
    assert e.value.name == status, str(e.value)


def test_rejects_bad_graphs():
    two = I.from_edges(4, [(0, 1), (2, 3)])                   # two components
    _expect("LAP_ERR_DISCONNECTED", lambda: LapGraph(two.row_ptr, two.col).set_root(0))
    rp = np.array([0, 1, 1], dtype=np.int32)                  # arc 0->1 without 1->0
    _expect("LAP_ERR_NOT_SYMMETRIC", lambda: LapGraph(rp, np.array([1], dtype=np.int32)))
    rp = np.array([0, 2, 3], dtype=np.int32)                  # self-loop at 0
    _expect("LAP_ERR_SELF_LOOP", lambda: LapGraph(rp, np.array([0, 1, 0], dtype=np.int32)))
    k = I.complete(4)
    col = k.col.copy()
    col[[0, 1]] = col[[1, 0]]                                 # unsorted row 0
    _expect("LAP_ERR_BAD_CSR", lambda: LapGraph(k.row_ptr, col))
    col = k.col.copy()
    col[0] = 7                                                # out of range
    _expect("LAP_ERR_BAD_CSR", lambda: LapGraph(k.row_ptr, col))
    _expect("LAP_ERR_INVALID_ARG", lambda: LapGraph(np.array([0, 0], dtype=np.int32), np.array([], dtype=np.int32)))


def test_seed_change_and_no_samples_are_rejected():
    g = I.cycle(10)
    G = LapGraph(g.row_ptr, g.col)
    try:
        _expect("LAP_ERR_NO_ROOT", lambda: G.sample(1, 1))
        G.set_root(0)
        _expect("LAP_ERR_NO_SAMPLES", lambda: G.kemeny())
        G.sample(3, 5)
        _expect("LAP_ERR_INVALID_ARG", lambda: G.sample(3, 6))
        G.sample(3, 5)
        assert G.counts()[2][0] == 6
    finally:
        G.close()


def test_step_budget_is_reported_and_cleared():
    """A path rooted at an end needs about n^2 steps per sample; a budget of
    100 steps must stop the kernel with LAP_ERR_STEP_LIMIT (no hang, no
    fault), and lap_set_root must clear the error."""
    g = I.path(400)
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=64 * 8 * g.n)
    try:
        G.set_option(LAP_OPT_STEP_LIMIT, 100)
        G.set_root(0)
        G.sample(20, 1)
        _expect("LAP_ERR_STEP_LIMIT", lambda: G.sync())
        _expect("LAP_ERR_STEP_LIMIT", lambda: G.kemeny())       # sticky
        G.set_option(LAP_OPT_STEP_LIMIT, 0)
        G.set_root(0)
        G.sample(4, 1)
        c1, _, s = G.counts()
        c = oracle.sample(g.row_ptr, g.col, 0, 1, 0, 4)
        assert np.array_equal(c1, c.cnt1) and int(s[1]) == c.sum_y1
    finally:
        G.close()


# ------------------------------------------------------------- full size

@pytest.fixture(scope="module")
def ba_1m():
    return I.ba_1m()


@pytest.mark.parametrize("kernel", [1, 2], ids=["wide", "compact"])
def test_full_size_ba_counts_small_omega(ba_1m, kernel):
    """The 10^6-node Barabasi-Albert workload graph: all counts bit-exact for 48 samples."""
    g = ba_1m
    r = gpu_run(g, 7, 48, kernel=kernel)
    c = oracle_run(g, r["v"], 7, 48, threads=8)
    assert_parity(g, r, c, 48)


def test_full_size_ba_bench_launch_sampled(ba_1m):
    """The benchmark's launch (default workspace, all slots busy, several
    samples per slot): per-sample Y1/Y2 of sampled ids against the oracle one
    by one, plus invariants that hold at any size (sum of visits = sum of Y1,
    every non-root node visited at least once per sample)."""
    g = ba_1m
    G = LapGraph(g.row_ptr, g.col)
    try:
        v = G.set_root()
        assert G.stat(LAP_STAT_KERNEL) == 2
        omega = int(min(2 * G.slots + 37, 400000))
        y1, y2 = G.sample_trace(omega, 2024)
        c1, c2, s = G.counts()
        assert G.stat(LAP_STAT_FALLBACKS) == 0
        y1 = y1.cpu().numpy().astype(np.uint64)
        y2 = y2.cpu().numpy().astype(np.uint64)
    finally:
        G.close()
    assert int(s[0]) == omega and int(s[1]) == int(y1.sum()) and int(s[2]) == int(y2.sum())
    assert int(c1.sum()) == int(s[1])
    mask = np.ones(g.n, bool)
    mask[v] = False
    assert c1[v] == 0 and np.all(c1[mask] >= omega)
    ids = np.unique(np.linspace(0, omega - 1, 12).astype(np.int64))
    for i in ids:
        c = oracle.sample(g.row_ptr, g.col, v, 2024, int(i), 1)
        assert c.y1[0] == y1[i] and c.y2[0] == y2[i], i


def test_small_workload_accuracy():
    """Erdos-Renyi G(1000, 0.01): estimates from 10^4 samples against the dense
    FP64 pseudo-inverse (loose bound; the time-to-1e-2 search is in bench.py)."""
    import oracle.dense as D
    g = I.er_1000()
    r = gpu_run(g, 1, 10000)
    ec = D.ecc(g.n, g.row_ptr, g.col)
    kc = D.kemeny(g.n, g.row_ptr, g.col)
    assert np.max(np.abs(r["ecc"] - ec) / ec) < 0.06
    assert abs(r["kc"] - kc) / kc < 0.02


def test_sharded_ranges_merge_with_set_counts():
    """Two handles draw disjoint sample-id ranges (LAP_OPT_CURSOR), their
    counts are summed on the host and loaded into a third handle with
    lap_set_counts: ECC and Kemeny equal, bit for bit, those of one handle
    that drew every id; the totals equal the oracle's."""
    from paper_2311_10290_gb300.lap import LAP_OPT_CURSOR, LapError, LapGraph
    from paper_2311_10290_gb300.shard import id_range
    g = I.ba(3000, 4, seed=12)
    total, seed = 900, 41
    parts = []
    for r in range(2):
        first, count = id_range(r, 2, total)
        G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 26)
        try:
            G.set_root()
            G.set_option(LAP_OPT_CURSOR, first)
            G.sample(count, seed)
            parts.append(G.counts())
        finally:
            G.close()
    c1 = parts[0][0] + parts[1][0]
    c2 = parts[0][1] + parts[1][1]
    s3 = np.array([total, int(parts[0][2][1]) + int(parts[1][2][1]), int(parts[0][2][2]) + int(parts[1][2][2])],
                  dtype=np.uint64)
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 26)
    H = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 26)
    try:
        v = G.set_root()
        G.set_counts(c1, c2, s3)
        H.set_root()
        H.sample(total, seed)
        assert np.array_equal(G.ecc(), H.ecc()) and G.kemeny() == H.kemeny()
        o = oracle.sample(g.row_ptr, g.col, v, seed, 0, total, keep_per_sample=False)
        assert np.array_equal(c1, o.cnt1) and np.array_equal(c2, o.cnt2)
        bad = c1.copy()
        bad[(v + 1) % g.n] = 0
        with pytest.raises(LapError, match="LAP_ERR_INVALID_ARG"):
            G.set_counts(bad, c2, s3)
    finally:
        G.close()
        H.close()
