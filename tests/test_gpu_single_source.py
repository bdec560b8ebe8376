"""Single-source rows of L_v^{-1} on the GPU (Section 4.2, "v-absorbed walk"
and "loop-erased walk" lemmas: started at a fixed s, the first absorbed walk,
or the loop-included path of the sample's own stacks, passes u on average
d_u (L_v^{-1})_{su} times).

Parity: with LAP_OPT_PATH_START = s the integer counts (Wilson visits, passes
of the walk from s, sum Y1, sum Y2) are bit-exact with oracle.sample(...,
path_start=s) in both walk modes, on both single-graph kernels (also when the
1-byte kernel withdraws samples and the 8-byte kernel re-runs them) and in
the batched sampler; lap_lv_row is cnt2[u] / (omega d_u), the same two IEEE
operations as the division below, so it is compared for equality."""
import numpy as np
import pytest

import oracle
from oracle import dense
from paper_2311_10290_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2311_10290_gb300.lap import (LAP_BOPT_LANES, LAP_BOPT_PATHS, LAP_BOPT_STACK,  # noqa: E402
                                        LAP_BSTAT_RERUNS, LAP_OPT_KERNEL, LAP_OPT_PATH_START, LAP_OPT_PATHS,
                                        LAP_OPT_CURSOR, LAP_OPT_SLOTS, LAP_OPT_STACK, LAP_STAT_FALLBACKS, LapBatch, LapError,
                                        LapGraph)


def row_from_counts(g, omega, cnt2):
    d = np.diff(g.row_ptr.astype(np.int64)).astype(np.float64)
    return cnt2.astype(np.float64) / (float(omega) * d)


def run_handle(g, root, s, seed, omega, kernel, paths, stack=None, slots=None):
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 26)
    try:
        G.set_option(LAP_OPT_KERNEL, kernel)
        if paths:
            G.set_option(LAP_OPT_PATHS, 1)
        if stack:
            G.set_option(LAP_OPT_STACK, stack)
        if slots:
            G.set_option(LAP_OPT_SLOTS, slots)
        G.set_option(LAP_OPT_PATH_START, s)
        v = G.set_root(root)
        G.sample(omega, seed)
        c1, c2, sums = G.counts()
        row = G.lv_row()
        kc = G.kemeny()
        fb = G.stat(LAP_STAT_FALLBACKS)
        with pytest.raises(LapError) as e:
            G.ecc()
        assert e.value.name == "LAP_ERR_INVALID_ARG"
        return v, c1, c2, sums, row, kc, fb
    finally:
        G.close()


CASES = [
    ("k4e", I.k4_minus_edge, 0, 2, 3000),
    ("path40_end", lambda: I.path(40), 0, 39, 300),
    ("er300", lambda: I.er(300, 0.02, seed=2), -1, 17, 800),
    ("ba2000", lambda: I.ba(2000, 3, seed=5), -1, 1999, 600),
]


@pytest.mark.parametrize("paths", [False, True], ids=["own_draws", "paths"])
@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("name,maker,root,s,omega", CASES, ids=[c[0] for c in CASES])
def test_fixed_start_counts_match_oracle(name, maker, root, s, omega, kernel, paths):
    g = maker()
    seed = 4242
    v, c1, c2, sums, row, kc, _ = run_handle(g, root, s, seed, omega, kernel, paths)
    c = oracle.sample(g.row_ptr, g.col, v, seed, 0, omega, keep_per_sample=False, paths=paths, path_start=s)
    assert np.array_equal(c1, c.cnt1)
    assert np.array_equal(c2, c.cnt2)
    assert int(sums[1]) == c.sum_y1 and int(sums[2]) == c.sum_y2
    assert np.array_equal(row, row_from_counts(g, omega, c.cnt2))
    assert row[v] == 0.0
    assert kc == pytest.approx((c.sum_y1 - c.sum_y2) / omega, rel=1e-15)


def test_fixed_start_with_withdrawn_samples_is_exact():
    """A 16-entry path stack cannot hold the loop-erased paths of a 200-node
    path rooted at one end: the 1-byte kernel withdraws those samples and
    the 8-byte kernel re-runs them, with the same fixed start."""
    g = I.path(200)
    for paths in (False, True):
        v, c1, c2, sums, row, _, fb = run_handle(g, 0, 150, 9, 64, 2, paths, stack=16, slots=8)
        assert fb > 0
        c = oracle.sample(g.row_ptr, g.col, v, 9, 0, 64, keep_per_sample=False, paths=paths, path_start=150)
        assert np.array_equal(c1, c.cnt1) and np.array_equal(c2, c.cnt2)
        assert int(sums[2]) == c.sum_y2
        assert np.array_equal(row, row_from_counts(g, 64, c.cnt2))


def test_row_estimates_resistance_and_lv_inverse_row():
    """Grounded at t, (L_t^{-1})_{ss} is the effective resistance between s
    and t: on a 31-node cycle R(s, t) = k (31 - k) / 31 at distance k.  Over
    40 GPU batches of 500 samples (disjoint ids), the mean row is within 6
    standard errors of the batch means (Student t, 39 degrees of freedom:
    P(|t| > 6) is about 5e-7 per node) of the dense row of L_t^{-1}."""
    g = I.cycle(31)
    t, s, k = 0, 9, 9
    batches, per = 40, 500
    rows = []
    for b in range(batches):
        G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 24)
        try:
            G.set_option(LAP_OPT_PATH_START, s)
            G.set_root(t)
            G.set_option(LAP_OPT_CURSOR, b * per)
            G.sample(per, 77)
            rows.append(G.lv_row())
        finally:
            G.close()
    rows = np.array(rows)
    want = dense.lv_inverse(g.n, g.row_ptr, g.col, t)[s]
    assert want[s] == pytest.approx(k * (31 - k) / 31.0, rel=1e-12)
    assert np.all(rows[:, t] == 0.0)
    m = rows.mean(axis=0)
    se = rows.std(axis=0, ddof=1) / np.sqrt(batches)
    live = np.arange(g.n) != t
    z = np.abs(m[live] - want[live]) / se[live]
    assert np.all(z < 6.0), (np.max(z), np.argmax(z))


def test_batch_fixed_starts_match_oracle():
    graphs = [I.er(300, 0.02, seed=2), I.ba(2000, 3, seed=5), I.path(200)]
    starts = [17, -1, 150]
    k, seed = 48, 13
    for paths in (0, 1):
        B = LapBatch([(g.row_ptr, g.col) for g in graphs], roots=[-1, -1, 0], workspace_bytes=1 << 24)
        try:
            B.set_option(LAP_BOPT_PATHS, paths)
            B.set_option(LAP_BOPT_STACK, 16)       # forces withdrawals on the path graph
            B.set_option(LAP_BOPT_LANES, 24)
            for j, s in enumerate(starts):
                B.set_path_start(j, s)
            B.run(k, seed)
            B.sync()
            assert B.stat(LAP_BSTAT_RERUNS) > 0
            for j, g in enumerate(graphs):
                v = int(B.roots[j])
                c1, c2, sums = B.counts(j)
                c = oracle.sample(g.row_ptr, g.col, v, seed, 0, k, keep_per_sample=False, paths=bool(paths),
                                  path_start=starts[j])
                assert np.array_equal(c1, c.cnt1), j
                assert np.array_equal(c2, c.cnt2), j
                assert int(sums[1]) == c.sum_y1 and int(sums[2]) == c.sum_y2, j
                assert np.array_equal(B.lv_row(j), row_from_counts(g, k, c.cnt2)), j
            # Back to the uniform start on the next run.
            B.set_path_start(0, -1)
            B.run(k, seed)
            c1, c2, _ = B.counts(0)
            v = int(B.roots[0])
            c = oracle.sample(graphs[0].row_ptr, graphs[0].col, v, seed, 0, k, keep_per_sample=False,
                              paths=bool(paths))
            assert np.array_equal(c2, c.cnt2)
        finally:
            B.close()


def test_fixed_start_option_is_validated():
    g = I.er(300, 0.02, seed=2)
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 22)
    try:
        for bad in (-2, g.n):
            with pytest.raises(LapError):
                G.set_option(LAP_OPT_PATH_START, bad)
        G.set_root(-1)
        G.sample(4, 1)
        with pytest.raises(LapError):            # only before the first sample
            G.set_option(LAP_OPT_PATH_START, 3)
    finally:
        G.close()
