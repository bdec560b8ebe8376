"""GPU parity of the batched persistent sampler (include/lap_batch.h) with the
oracle: every graph's integer counts bit-exact with oracle.sample for the
same root, seed and sample ids; ECC, (L^+)_uu and Kemeny within 1e-12 of
oracle.finalize and bit-identical to a single-graph handle; withdrawn
samples re-run exactly; results independent of lanes, claim size, order and
CUDA-graph replay; the autotuner's choice keeps the counts."""
import numpy as np
import pytest

import oracle
from paper_2311_10290_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2311_10290_gb300.lap import (LAP_BOPT_CLAIM, LAP_BOPT_LANES, LAP_BOPT_ORDER, LAP_BOPT_PATHS,  # noqa: E402
                                        LAP_BOPT_STACK,
                                        LAP_BSTAT_GRAPH_CAPTURES, LAP_BSTAT_RERUNS, LapBatch, LapError, LapGraph)


def mixed_graphs():
    """Uneven sizes and families; increasing n in the caller's order."""
    return [I.star(20), I.path(30), I.cycle(41), I.complete(12), I.er(200, 0.04, seed=3),
            I.ba(700, 3, seed=4), I.rmat(10, 6, seed=5), I.ba(2500, 5, seed=6), I.er(3000, 0.003, seed=7)]


def oracle_results(g, v, seed, k):
    c = oracle.sample(g.row_ptr, g.col, v, seed, 0, k, keep_per_sample=False)
    ld, ec, kc = oracle.finalize(g.row_ptr, v, k, c.cnt1, c.cnt2, c.sum_y1, c.sum_y2)
    return c, ld, ec, kc


def check_against_oracle(B, graphs, seed, k, ref=None):
    ecc = B.split(B.ecc())
    ld = B.split(B.ldiag())
    kc = B.kemeny()
    for j, g in enumerate(graphs):
        v = int(B.roots[j])
        c1, c2, sums = B.counts(j)
        c, ldo, eco, kco = ref[j] if ref else oracle_results(g, v, seed, k)
        assert np.array_equal(c1, c.cnt1), j
        assert np.array_equal(c2, c.cnt2), j
        assert int(sums[0]) == k and int(sums[1]) == c.sum_y1 and int(sums[2]) == c.sum_y2, j
        # (L^+)_uu = y1 - 2 y2 + lvv can cancel to near zero at small omega:
        # the bound is 1e-12 relative to the magnitude of its terms.
        d = np.diff(g.row_ptr.astype(np.int64)).astype(np.float64)
        scale = (c.cnt1.astype(np.float64) + 2.0 * c.cnt2.astype(np.float64)) / (k * d) + np.abs(ldo[v])
        assert np.all(np.abs(ld[j] - ldo) <= 1e-12 * scale), j
        np.testing.assert_allclose(ecc[j], eco, rtol=1e-12)
        assert kc[j] == pytest.approx(kco, rel=1e-12)


@pytest.mark.parametrize("order", [0, 1, 2], ids=["largest_first", "smallest_first", "given"])
@pytest.mark.parametrize("lanes,claim", [(64, 1), (160, 3), (0, 7)])
def test_batch_counts_match_oracle(order, lanes, claim):
    graphs = mixed_graphs()
    k, seed = 40, 11
    B = LapBatch([(g.row_ptr, g.col) for g in graphs], workspace_bytes=1 << 26)
    try:
        B.set_option(LAP_BOPT_ORDER, order)
        B.set_option(LAP_BOPT_LANES, lanes)
        B.set_option(LAP_BOPT_CLAIM, claim)
        B.run(k, seed)
        for j, g in enumerate(graphs):
            assert B.roots[j] == oracle.root_max_degree(g.row_ptr)
        check_against_oracle(B, graphs, seed, k)
    finally:
        B.close()


def test_batch_equals_single_graph_handles_bitwise():
    graphs = mixed_graphs()
    k, seed = 33, 5
    roots = [-1, 0, 7, 3, 10, -1, 2, -1, 100]
    B = LapBatch([(g.row_ptr, g.col) for g in graphs], roots=roots, workspace_bytes=1 << 26)
    try:
        B.run(k, seed)
        ecc = B.split(B.ecc())
        kc = B.kemeny()
        for j, g in enumerate(graphs):
            G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 24)
            try:
                v = G.set_root(roots[j])
                assert v == B.roots[j]
                G.sample(k, seed)
                assert np.array_equal(G.ecc(), ecc[j])
                assert G.kemeny() == kc[j]
            finally:
                G.close()
    finally:
        B.close()


def test_batch_withdrawn_samples_are_rerun_exactly():
    """A small path stack (64 entries after rounding the slot to 256 bytes)
    cannot hold the 199-node loop-erased path of a 200-node path rooted at one
    end, nor the long way round a 300-cycle: those samples are withdrawn and
    re-run with the 8-byte kernel."""
    graphs = [I.path(200), I.star(30), I.cycle(300), I.ba(400, 2, seed=1)]
    k, seed = 24, 3
    B = LapBatch([(g.row_ptr, g.col) for g in graphs], roots=[199, -1, 0, -1], workspace_bytes=1 << 24)
    try:
        B.set_option(LAP_BOPT_STACK, 16)
        B.set_option(LAP_BOPT_LANES, 20)
        B.run(k, seed)
        check_against_oracle(B, graphs, seed, k)
        assert B.stat(LAP_BSTAT_RERUNS) > 0
        # A second run on the same handle (slots hold 8-byte states after the re-run).
        B.run(k, seed + 1)
        check_against_oracle(B, graphs, seed + 1, k)
    finally:
        B.close()


def test_graph_replay_and_option_changes_keep_results():
    graphs = mixed_graphs()
    k, seed = 25, 8
    ref = [oracle_results(g, oracle.root_max_degree(g.row_ptr), seed, k) for g in graphs]
    B = LapBatch([(g.row_ptr, g.col) for g in graphs], workspace_bytes=1 << 26)
    try:
        B.run(k, seed)
        check_against_oracle(B, graphs, seed, k, ref)
        B.run(k, seed)                      # replay of the same CUDA graph
        check_against_oracle(B, graphs, seed, k, ref)
        assert B.stat(LAP_BSTAT_GRAPH_CAPTURES) == 1
        B.set_option(LAP_BOPT_CLAIM, 4)
        B.set_option(LAP_BOPT_LANES, 50)
        B.run(k, seed)
        check_against_oracle(B, graphs, seed, k, ref)
        assert B.stat(LAP_BSTAT_GRAPH_CAPTURES) == 2
        t = B.completion()
        assert np.all(t > 0) and np.all(t < 60)
    finally:
        B.close()


def test_autotune_then_run_is_exact():
    graphs = mixed_graphs()
    k, seed = 64, 21
    B = LapBatch([(g.row_ptr, g.col) for g in graphs], workspace_bytes=1 << 27)
    try:
        table = B.autotune(k, seed, window_ms=20.0)
        assert len(table) == 6
        assert all(r[2] > 0 for r in table)
        assert B.stat(LAP_BSTAT_GRAPH_CAPTURES) == 0
        B.run(k, seed)
        check_against_oracle(B, graphs, seed, k)
    finally:
        B.close()


def test_batch_rejects_bad_graphs():
    good = I.ba(100, 2, seed=1)
    two = I.from_edges(4, np.array([[0, 1], [2, 3]], dtype=np.int64))
    with pytest.raises(LapError, match="graph 1: .*not connected"):
        LapBatch([(good.row_ptr, good.col), (two.row_ptr, two.col)], workspace_bytes=1 << 22)
    rp = np.array([0, 1, 1], dtype=np.int32)
    col = np.array([1], dtype=np.int32)
    with pytest.raises(LapError, match="LAP_ERR_NOT_SYMMETRIC"):
        LapBatch([(good.row_ptr, good.col), (rp, col)], workspace_bytes=1 << 22)
    with pytest.raises(LapError, match="LAP_ERR_INVALID_ARG"):
        LapBatch([(good.row_ptr, good.col)], roots=[500], workspace_bytes=1 << 22)


def test_uneven_batch_sampled_parity_and_invariants():
    """Forty graphs of the uneven recipe (ER/BA/R-MAT by seed mod 3, n
    log-uniform, average degree in [4, 32]) at 512 samples, lanes chosen by
    the autotuner: the five smallest graphs bit-exact with the oracle, and on
    every graph the identities that hold at any size: cnt1[v] = 0,
    cnt1[u] >= omega for u != v, sum_u cnt1[u] = sum Y1, and cnt2[v] = 0."""
    spec = I.batch_spec(count=40, n_lo=1_000, n_hi=60_000, seed0=7000)
    graphs = [I.batch_graph(*s) for s in spec]
    k, seed = 512, 77
    B = LapBatch([(g.row_ptr, g.col) for g in graphs])
    try:
        B.autotune(k, seed, window_ms=30.0)
        B.run(k, seed)
        B.sync()
        small = np.argsort([g.n for g in graphs])[:5]
        for j in small:
            v = int(B.roots[j])
            c = oracle.sample(graphs[j].row_ptr, graphs[j].col, v, seed, 0, k, keep_per_sample=False)
            c1, c2, sums = B.counts(int(j))
            assert np.array_equal(c1, c.cnt1) and np.array_equal(c2, c.cnt2)
            assert int(sums[1]) == c.sum_y1 and int(sums[2]) == c.sum_y2
        for j, g in enumerate(graphs):
            v = int(B.roots[j])
            c1, c2, sums = B.counts(j)
            assert c1[v] == 0 and c2[v] == 0
            mask = np.ones(g.n, bool)
            mask[v] = False
            assert np.all(c1[mask] >= k)
            assert int(c1.sum(dtype=np.uint64)) == int(sums[1])
        kc = B.kemeny()
        assert np.all(np.isfinite(kc)) and np.all(kc > 0)
        t = B.completion()
        assert np.all(t > 0)
    finally:
        B.close()


def test_uneven_batch_full_recipe_sampled_parity():
    """The full uneven workload (512 graphs, n log-uniform in [1e3, 1e6],
    4096 samples each) in the launch the benchmark times (autotuned lanes and
    claim): the three smallest graphs bit-exact with the oracle; the
    any-size identities on every graph."""
    spec = I.batch_spec()
    graphs = I.batch_graphs(spec)
    k, seed = 4096, 1
    B = LapBatch([(g.row_ptr, g.col) for g in graphs])
    try:
        B.autotune(k, seed)
        B.run(k, seed)
        B.sync()
        small = np.argsort([g.n for g in graphs])[:3]
        for j in small:
            v = int(B.roots[j])
            c = oracle.sample(graphs[j].row_ptr, graphs[j].col, v, seed, 0, k, keep_per_sample=False)
            c1, c2, sums = B.counts(int(j))
            assert np.array_equal(c1, c.cnt1) and np.array_equal(c2, c.cnt2)
            assert int(sums[1]) == c.sum_y1 and int(sums[2]) == c.sum_y2
        for j in range(len(graphs)):
            v = int(B.roots[j])
            c1, c2, sums = B.counts(j)
            assert c1[v] == 0 and c2[v] == 0
            assert int(c1.sum(dtype=np.uint64)) == int(sums[1])
            assert int(np.delete(c1, v).min()) >= k
    finally:
        B.close()


def test_many_roots_of_one_graph_share_the_csr():
    """A landmark study (Section 6): one graph, many roots, passed as the same
    arrays, so the batch keeps one copy of the CSR.  Every root's counts equal
    the oracle's; sum Y1 / omega estimates Tr((I - P_v)^{-1}) (dense check
    within 6 standard errors)."""
    import oracle.dense as D
    g = I.ba(1500, 3, seed=21)
    deg = np.diff(g.row_ptr)
    roots = [int(np.argmax(deg)), 0, 17, int(np.argmin(deg)), 700, 1499]
    k, seed = 300, 13
    B = LapBatch([(g.row_ptr, g.col)] * len(roots), roots=roots, workspace_bytes=1 << 26)
    try:
        B.run(k, seed)
        tr = B.mean_wilson_steps()
        for j, v in enumerate(roots):
            c = oracle.sample(g.row_ptr, g.col, v, seed, 0, k)
            c1, c2, sums = B.counts(j)
            assert np.array_equal(c1, c.cnt1) and np.array_equal(c2, c.cnt2) and int(sums[1]) == c.sum_y1
            lv = D.lv_inverse(g.n, g.row_ptr, g.col, v)
            exact = float(np.sum(np.diag(lv) * deg))         # Tr((I - P_v)^{-1}) = sum_u d_u (L_v^{-1})_uu
            se = np.std(c.y1.astype(np.float64)) / np.sqrt(k)
            assert abs(tr[j] - exact) < 6 * se + 1e-9, (v, tr[j], exact, se)
        assert np.argmin(tr) == 0                     # the hub is the cheapest root
    finally:
        B.close()


def test_kirchhoff_and_rw_betweenness_match_oracle():
    import oracle.dense as D
    graphs = [I.er(300, 0.03, seed=2), I.ba(900, 4, seed=3)]
    k, seed = 500, 9
    B = LapBatch([(g.row_ptr, g.col) for g in graphs], workspace_bytes=1 << 26)
    try:
        B.run(k, seed)
        kf_b = B.kirchhoff()
    finally:
        B.close()
    for j, g in enumerate(graphs):
        G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 24)
        try:
            v = G.set_root()
            G.sample(k, seed)
            kf = G.kirchhoff()
            cb = G.rw_betweenness()
            cb_dev = G.rw_betweenness(torch.empty(g.n, dtype=torch.float64, device="cuda")).cpu().numpy()
        finally:
            G.close()
        c = oracle.sample(g.row_ptr, g.col, v, seed, 0, k, keep_per_sample=False)
        ld, _, _ = oracle.finalize(g.row_ptr, v, k, c.cnt1, c.cnt2, c.sum_y1, c.sum_y2)
        tr, cbo = D.from_ldiag(ld)
        assert kf == pytest.approx(tr, rel=1e-12) and kf == kf_b[j]
        np.testing.assert_allclose(cb, cbo, rtol=1e-12)
        assert np.array_equal(cb, cb_dev)


def test_batch_loop_included_paths_match_oracle():
    graphs = mixed_graphs() + [I.path(256)]
    roots = [-1] * (len(graphs) - 1) + [255]
    k, seed = 30, 4
    B = LapBatch([(g.row_ptr, g.col) for g in graphs], roots=roots, workspace_bytes=1 << 26)
    try:
        B.set_option(LAP_BOPT_PATHS, 1)
        B.set_option(LAP_BOPT_LANES, 96)
        B.run(k, seed)
        for j, g in enumerate(graphs):
            v = int(B.roots[j])
            c = oracle.sample(g.row_ptr, g.col, v, seed, 0, k, keep_per_sample=False, paths=True)
            c1, c2, sums = B.counts(j)
            assert np.array_equal(c1, c.cnt1) and np.array_equal(c2, c.cnt2), j
            assert int(sums[1]) == c.sum_y1 and int(sums[2]) == c.sum_y2, j
    finally:
        B.close()
