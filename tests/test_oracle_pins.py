"""Pins for the CPU oracle: each test ties the oracle to something other than
itself (a value the paper prints, a closed form, a theorem that can be checked
by enumeration, an exact special case, or the estimand's expectation).

Runs on CPU only (no GPU marker)."""
import itertools

import numpy as np
import pytest
from scipy import stats

import oracle
import oracle.dense as D
from _golden import read_kv, read_rows
from paper_2311_10290_gb300 import inputs as I


# --------------------------------------------------------------------- Philox

def test_philox_known_answers():
    """Philox4x32-10 against the published known-answer vectors."""
    for row in read_rows("philox4x32_10_kat.txt"):
        w = [int(x, 16) for x in row]
        got = oracle.philox_block(w[0:4], w[4:6])
        assert [int(x) for x in got] == w[6:10]


# ------------------------------------------------- paper's worked example

def _k4e():
    return I.k4_minus_edge()


def test_k4e_pinv_values_printed_in_paper():
    kv = read_kv("k4e_worked_example.txt")
    g = _k4e()
    lp = D.pinv_laplacian(g.n, g.row_ptr, g.col)
    assert lp[0, 0] == pytest.approx(kv["ldag_vv"], abs=1e-14)
    assert lp[0, 3] == pytest.approx(kv["ldag_v_other_deg2"], abs=1e-14)
    # Edge currents for 1/n injected everywhere and 1 extracted at v = node 0.
    b = np.full(4, 0.25)
    b[0] -= 1.0
    x = lp @ b
    cur = sorted(abs(x[u] - x[w]) for u in range(4) for w in g.col[g.row_ptr[u]:g.row_ptr[u + 1]] if u < w)
    assert np.allclose(cur, sorted(kv["edge_currents"]), atol=1e-14)
    assert sum(c * c for c in cur) == pytest.approx(kv["ldag_vv"], abs=1e-14)


def test_k4e_weighted_voltage_sum():
    """(1/2m) d_v^T L_v^{-1} d_v = 3.4 for v a degree-2 node (the paper's own sum)."""
    kv = read_kv("k4e_worked_example.txt")
    g = _k4e()
    e = D.expectations(g.n, g.row_ptr, g.col, 0)
    assert e["y2"] == pytest.approx(kv["weighted_voltage_sum"], abs=1e-13)
    assert e["y2"] == pytest.approx((32 * 3 + 32 * 3 + 40 * 2) / 80, abs=1e-13)


# ------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [3, 4, 5, 8, 13])
def test_kemeny_closed_forms(n):
    """kappa(K_n) = (n-1)^2/n, kappa(C_n) = (n^2-1)/6, kappa(P_n) = (2(n-1)^2+1)/6,
    kappa(S_n) = n - 3/2."""
    cases = [(I.complete(n), (n - 1) ** 2 / n), (I.cycle(n), (n * n - 1) / 6),
             (I.path(n), (2 * (n - 1) ** 2 + 1) / 6), (I.star(n), n - 1.5)]
    for g, want in cases:
        assert D.kemeny(g.n, g.row_ptr, g.col) == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("n", [3, 6, 11])
def test_ecc_complete_graph(n):
    g = I.complete(n)
    assert np.allclose(D.ecc(g.n, g.row_ptr, g.col), n / 2, rtol=1e-12)


@pytest.mark.parametrize("n", [5, 9])
def test_resistance_path_and_cycle(n):
    """r(s,t) = L+_ss + L+_tt - 2 L+_st (Section 2): |i-j| on a path, k(n-k)/n on a cycle."""
    for g, want in [(I.path(n), lambda i, j: abs(i - j)),
                    (I.cycle(n), lambda i, j: (abs(i - j) * (n - abs(i - j))) / n)]:
        lp = D.pinv_laplacian(g.n, g.row_ptr, g.col)
        for i in range(n):
            for j in range(n):
                r = lp[i, i] + lp[j, j] - 2 * lp[i, j]
                assert r == pytest.approx(want(i, j), abs=1e-11)


def test_path_rooted_at_end_trace():
    """Tr((I - P_v)^{-1}) = (n-1)^2 on a path rooted at an end."""
    for n in [4, 7, 12]:
        g = I.path(n)
        assert D.expectations(g.n, g.row_ptr, g.col, 0)["y1"] == pytest.approx((n - 1) ** 2, rel=1e-12)


# ------------------------------------------------------------ identities

def _small_graphs():
    return [I.er(40, 0.12, seed=3), I.ba(35, 2, seed=5), I.rmat(6, 4, seed=7), _k4e(), I.cycle(9)]


def test_theorem1_elementwise_matches_pinv():
    """L^+ from L_v^{-1} (Thm 1 and its element-wise cases) equals the
    eigendecomposition pseudo-inverse, for several landmarks."""
    for g in _small_graphs():
        lp = D.pinv_laplacian(g.n, g.row_ptr, g.col)
        for v in {0, g.n // 2, g.n - 1, oracle.root_max_degree(g.row_ptr)}:
            li = D.lv_inverse(g.n, g.row_ptr, g.col, v)
            assert np.allclose(D.ldag_from_lv(g.n, li, v), lp, atol=1e-11)


def test_kemeny_lemma():
    """Tr(calL^+) = Tr((I-P_v)^{-1}) - (1/2m) d_v^T L_v^{-1} d_v for every v (Section 5 lemma)."""
    for g in _small_graphs():
        kc = D.kemeny(g.n, g.row_ptr, g.col)
        for v in [0, g.n - 1, oracle.root_max_degree(g.row_ptr)]:
            e = D.expectations(g.n, g.row_ptr, g.col, v)
            assert e["y1"] - e["y2"] == pytest.approx(kc, rel=1e-10)


def test_hitting_times_mean_is_weighted_voltage_sum():
    """sum_u pi(u) h(u, v) = (1/2m) d^T L_v^{-1} d (Section 5, LEWalk for KC)."""
    for g in _small_graphs():
        v = oracle.root_max_degree(g.row_ptr)
        h = D.hitting_times_to(g.n, g.row_ptr, g.col, v)
        pi = g.degree / g.degree.sum()
        assert float(pi @ h) == pytest.approx(D.expectations(g.n, g.row_ptr, g.col, v)["y2"], rel=1e-11)


# --------------------------------------------------- Matrix-Tree / Wilson

def _edges(g):
    return [(u, int(w)) for u in range(g.n) for w in g.col[g.row_ptr[u]:g.row_ptr[u + 1]] if u < w]


def _spanning_trees(g):
    edges = _edges(g)
    trees = []
    for sub in itertools.combinations(range(len(edges)), g.n - 1):
        par = list(range(g.n))

        def find(x):
            while par[x] != x:
                x = par[x]
            return x
        ok = True
        for k in sub:
            a, b = find(edges[k][0]), find(edges[k][1])
            if a == b:
                ok = False
                break
            par[a] = b
        if ok:
            trees.append(frozenset(edges[k] for k in sub))
    return trees


def _tree_edges(parent, v):
    return frozenset((min(u, int(p)), max(u, int(p))) for u, p in enumerate(parent) if u != v)


@pytest.mark.parametrize("name,maker,count", [("K4-e", _k4e, 8), ("K4", lambda: I.complete(4), 16),
                                              ("C5", lambda: I.cycle(5), 5)])
def test_matrix_tree_and_uniform_trees(name, maker, count):
    """Number of spanning trees = det(L_v) (Matrix-Tree theorem), and the
    oracle's Wilson trees are uniform over them (chi-square)."""
    g = maker()
    trees = _spanning_trees(g)
    assert len(trees) == count
    lap = D.laplacian(g.n, g.row_ptr, g.col)
    assert round(np.linalg.det(lap[1:, 1:])) == count
    if name == "K4-e":
        assert count == read_kv("k4e_worked_example.txt")["spanning_trees"]
    index = {t: k for k, t in enumerate(trees)}
    omega = 4000 * count
    c = oracle.sample(g.row_ptr, g.col, 0, 99, 0, omega, keep_tree=True)
    hist = np.zeros(count)
    for parent in c.tree:
        hist[index[_tree_edges(parent, 0)]] += 1
    chi = stats.chisquare(hist)
    assert chi.pvalue > 1e-6, (hist, chi)


def test_trees_are_spanning_trees_rooted_at_v():
    g = I.er(60, 0.1, seed=11)
    v = oracle.root_max_degree(g.row_ptr)
    c = oracle.sample(g.row_ptr, g.col, v, 5, 0, 50, keep_tree=True)
    for parent in c.tree:
        assert parent[v] == -1
        for u in range(g.n):
            if u == v:
                continue
            assert parent[u] in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]
            x, steps = u, 0
            while x != v:
                x = parent[x]
                steps += 1
                assert steps <= g.n


# ----------------------------------------- order independence (Section 3.4)

@pytest.mark.parametrize("g", [I.er(80, 0.06, seed=2), I.ba(120, 2, seed=4), I.path(30), _k4e()],
                         ids=["er", "ba", "path", "k4e"])
def test_counts_do_not_depend_on_start_order(g):
    """With draws keyed by (node, draw index), any start order gives the same
    stacks, hence the same visits, tree and walk lengths (Fig. 1)."""
    v = oracle.root_max_degree(g.row_ptr)
    base = oracle.sample(g.row_ptr, g.col, v, 2024, 10, 40, keep_tree=True)
    rng = np.random.default_rng(0)
    for _ in range(3):
        order = rng.permutation(g.n).astype(np.int32)
        other = oracle.sample(g.row_ptr, g.col, v, 2024, 10, 40, order=order, keep_tree=True)
        assert np.array_equal(base.cnt1, other.cnt1)
        assert np.array_equal(base.cnt2, other.cnt2)
        assert np.array_equal(base.y1, other.y1)
        assert np.array_equal(base.y2, other.y2)
        assert np.array_equal(base.tree, other.tree)


@pytest.mark.parametrize("g", [I.er(80, 0.06, seed=2), I.ba(150, 3, seed=8), I.cycle(17), I.rmat(7, 6, seed=1)],
                         ids=["er", "ba", "cycle", "rmat"])
def test_cycle_popping_matches_sequential_walks(g):
    """visits(u) = pops(u) + 1: round-wise cycle popping on the stacks gives the
    sequential run's counts, Y1 and tree exactly."""
    v = oracle.root_max_degree(g.row_ptr)
    seq = oracle.sample(g.row_ptr, g.col, v, 77, 0, 30, keep_tree=True)
    cnt1, y1, tree = oracle.cyclepop(g.row_ptr, g.col, v, 77, 0, 30, keep_tree=True)
    assert np.array_equal(seq.cnt1, cnt1)
    assert np.array_equal(seq.y1, y1)
    assert np.array_equal(seq.tree, tree)


# ------------------------------------------------------- exact special cases

@pytest.mark.parametrize("n", [2, 5, 40])
def test_star_rooted_at_hub_exact_counts(n):
    """Star rooted at its hub: every leaf is visited exactly once per run
    (Y1 = n-1), a walk from a leaf passes it once and is absorbed, and the
    pi-start walk has length 0 or 1 with probability 1/2 each."""
    g = I.star(n)
    omega = 3000
    c = oracle.sample(g.row_ptr, g.col, 0, 3, 0, omega)
    assert np.all(c.cnt1[1:] == omega) and c.cnt1[0] == 0
    assert np.all(c.y1 == n - 1)
    assert c.cnt2[0] == 0 and np.all(c.cnt2 <= omega) and int(c.cnt2.sum()) <= omega
    assert set(np.unique(c.y2)) <= {0, 1}
    assert abs(c.y2.mean() - 0.5) < 6 * 0.5 / np.sqrt(omega)
    assert abs(c.cnt2.sum() / omega - (n - 1) / n) < 6 * np.sqrt(1.0 / omega)


@pytest.mark.parametrize("n", [3, 6, 10])
def test_finalize_on_exact_star_expectations(n):
    """Counts equal to their expectations (omega a multiple of 2n) must give the
    dense L+ diagonal, the dense ECC and kappa(S_n) = n - 3/2."""
    g = I.star(n)
    omega = 2 * n * 7
    cnt1 = np.array([0] + [omega] * (n - 1), dtype=np.uint64)
    cnt2 = np.array([0] + [omega // n] * (n - 1), dtype=np.uint64)
    ld, ec, kc = oracle.finalize(g.row_ptr, 0, omega, cnt1, cnt2, omega * (n - 1), omega // 2)
    assert np.allclose(ld, np.diag(D.pinv_laplacian(g.n, g.row_ptr, g.col)), rtol=1e-13, atol=1e-15)
    assert np.allclose(ec, D.ecc(g.n, g.row_ptr, g.col), rtol=1e-13)
    assert kc == pytest.approx(n - 1.5, rel=1e-14)


def test_finalize_on_exact_k4e_expectations():
    """K4-e, v = 0: E[visits] = (0, 15/8, 15/8, 2), E[passes] = (0, 9/8, 9/8, 1),
    E[Y1] = 23/4, E[Y2] = 17/5; with omega = 40 these are integers and the
    finalize must return L+ diag (5/16, 3/16, 3/16, 5/16) and kappa = 2.35."""
    g = _k4e()
    e = D.expectations(g.n, g.row_ptr, g.col, 0)
    omega = 40
    cnt1 = np.rint(e["visits"] * omega).astype(np.uint64)
    cnt2 = np.rint(e["passes"] * omega).astype(np.uint64)
    assert np.allclose(cnt1, e["visits"] * omega, atol=1e-9) and np.allclose(cnt2, e["passes"] * omega, atol=1e-9)
    y1, y2 = round(e["y1"] * omega), round(e["y2"] * omega)
    ld, ec, kc = oracle.finalize(g.row_ptr, 0, omega, cnt1, cnt2, y1, y2)
    kv = read_kv("k4e_worked_example.txt")
    assert ld[0] == pytest.approx(kv["ldag_vv"], abs=1e-15)
    assert np.allclose(ld, [5 / 16, 3 / 16, 3 / 16, 5 / 16], atol=1e-15)
    assert np.allclose(ec, D.ecc(g.n, g.row_ptr, g.col), rtol=1e-13)
    assert kc == pytest.approx(D.kemeny(g.n, g.row_ptr, g.col), rel=1e-13)


# ------------------------------------------------ means match the estimand

def _batch_means(g, v, batches, per, paths=False):
    c1, c2, y1, y2 = [], [], [], []
    for b in range(batches):
        c = oracle.sample(g.row_ptr, g.col, v, 4242, b * per, per, paths=paths)
        c1.append(c.cnt1 / per)
        c2.append(c.cnt2 / per)
        y1.append(c.sum_y1 / per)
        y2.append(c.sum_y2 / per)
    return [np.array(x) for x in (c1, c2, y1, y2)]


def _check(mean_batches, expected):
    m = mean_batches.mean(axis=0)
    se = mean_batches.std(axis=0, ddof=1) / np.sqrt(mean_batches.shape[0])
    z = np.abs(m - expected) / np.maximum(se, 1e-12)
    exact = se < 1e-12
    assert np.all(z[~exact] < 6.0), (m, expected, se)
    assert np.allclose(m[exact], np.atleast_1d(expected)[exact] if np.ndim(expected) else expected, atol=1e-9)


@pytest.mark.parametrize("g,root", [(_k4e(), 0), (I.er(30, 0.2, seed=1), None), (I.ba(40, 2, seed=3), None),
                                    (I.path(6), 0), (I.cycle(7), 3), (I.rmat(5, 4, seed=2), None)],
                         ids=["k4e", "er", "ba", "path", "cycle", "rmat"])
def test_sample_means_match_dense_expectations(g, root):
    """Lemma (LE walk): E[visits(u)] = d_u (L_v^{-1})_uu; Lemma (sample the
    paths): E[passes(u)] = d_u (1/n) e_u^T L_v^{-1} 1; Alg. 4: E[Y1] =
    Tr((I-P_v)^{-1}), E[Y2] = (1/2m) d^T L_v^{-1} d."""
    v = oracle.root_max_degree(g.row_ptr) if root is None else root
    e = D.expectations(g.n, g.row_ptr, g.col, v)
    c1, c2, y1, y2 = _batch_means(g, v, 24, 1500)
    _check(c1, e["visits"])
    _check(c2, e["passes"])
    _check(y1[:, None], np.array([e["y1"]]))
    _check(y2[:, None], np.array([e["y2"]]))


@pytest.mark.parametrize("g,root", [(_k4e(), 0), (I.er(30, 0.2, seed=1), None), (I.ba(40, 2, seed=3), None),
                                    (I.path(6), 0), (I.cycle(7), 3)],
                         ids=["k4e", "er", "ba", "path", "cycle"])
def test_loop_included_paths_have_the_walk_expectations(g, root):
    """Section 4.2 ("loop-erased walk" lemma, "sample the paths") and
    Section 5.2: the loop-included path of the sample's stacks from a uniform
    (or pi-distributed) start has the law of a v-absorbed walk from it, so
    the counts keep the expectations of the online walks."""
    v = oracle.root_max_degree(g.row_ptr) if root is None else root
    e = D.expectations(g.n, g.row_ptr, g.col, v)
    c1, c2, y1, y2 = _batch_means(g, v, 24, 1500, paths=True)
    _check(c1, e["visits"])
    _check(c2, e["passes"])
    _check(y1[:, None], np.array([e["y1"]]))
    _check(y2[:, None], np.array([e["y2"]]))


def _uniform_start(n, seed, i):
    """Start node of sample i's uniform walk: counter (0, 0, i, 1), high 64
    bits of R64 * n (the same reading as the sampler's)."""
    blk = oracle.philox_block([0, 0, i, 1], [seed & 0xFFFFFFFF, seed >> 32])
    r = int(blk[0]) | (int(blk[1]) << 32)
    return (r * n) >> 64


def test_loop_included_path_is_the_first_walk_from_its_start():
    """By the stack representation (Fig. 1), the loop-included path from s
    is exactly the walk Wilson's algorithm takes from s when s is the first
    start: the same draws (u, j) in the same order.  So its length equals Y1
    of a run whose only start is s, and no node is left more often than the
    full run draws from it."""
    g = I.ba(60, 2, seed=4)
    v = oracle.root_max_degree(g.row_ptr)
    seed = 77
    checked = 0
    for i in range(40):
        s = _uniform_start(g.n, seed, i)
        if s == v:
            continue
        full = oracle.sample(g.row_ptr, g.col, v, seed, i, 1, paths=True)
        first = oracle.sample(g.row_ptr, g.col, v, seed, i, 1, order=np.array([s], dtype=np.int32), paths=True)
        assert int(full.cnt2.sum()) == int(first.y1[0])             # path length = first walk's steps
        assert np.array_equal(first.cnt1, full.cnt2)                 # passes per node = that walk's visits
        assert np.all(full.cnt2 <= full.cnt1)                        # a prefix of every node's stack
        assert full.y2[0] <= full.y1[0]
        checked += 1
    assert checked > 30


def test_loop_included_paths_reduce_the_kemeny_variance():
    """Sharing the stacks with the Wilson run correlates Y2 with Y1: on
    G(200, 0.05) the per-sample variance of Y1 - Y2 drops by more than half."""
    g = I.er(200, 0.05, seed=0)
    v = oracle.root_max_degree(g.row_ptr)
    a = oracle.sample(g.row_ptr, g.col, v, 3, 0, 6000)
    b = oracle.sample(g.row_ptr, g.col, v, 3, 0, 6000, paths=True)
    assert np.array_equal(a.cnt1, b.cnt1) and np.array_equal(a.y1, b.y1)    # the Wilson part is shared
    va = np.var(a.y1.astype(np.float64) - a.y2)
    vb = np.var(b.y1.astype(np.float64) - b.y2)
    assert vb < 0.5 * va, (vb, va)


def test_estimates_converge_on_small_er():
    """ECC and KC from the oracle's counts approach the dense values (the
    accuracy target of the small workload, checked loosely)."""
    g = I.er(200, 0.05, seed=0)
    v = oracle.root_max_degree(g.row_ptr)
    c = oracle.sample(g.row_ptr, g.col, v, 1, 0, 20000, keep_per_sample=False)
    ld, ec, kc = oracle.finalize(g.row_ptr, v, c.omega, c.cnt1, c.cnt2, c.sum_y1, c.sum_y2)
    assert np.max(np.abs(ec - D.ecc(g.n, g.row_ptr, g.col)) / D.ecc(g.n, g.row_ptr, g.col)) < 0.03
    assert abs(kc - D.kemeny(g.n, g.row_ptr, g.col)) / D.kemeny(g.n, g.row_ptr, g.col) < 0.01
    lp = D.pinv_laplacian(g.n, g.row_ptr, g.col)
    assert np.sum(ld) == pytest.approx(np.trace(lp), rel=0.01)     # Kirchhoff index Tr(L+)


# ----------------------------------------------------------- step budget

def test_step_budget_reports_overrun():
    g = I.path(40)
    with pytest.raises(RuntimeError):
        oracle.sample(g.row_ptr, g.col, 0, 1, 0, 2, max_steps=10)
    oracle.sample(g.row_ptr, g.col, 0, 1, 0, 2, max_steps=10 ** 7)


def test_thread_split_is_exact():
    g = I.ba(500, 3, seed=9)
    v = oracle.root_max_degree(g.row_ptr)
    a = oracle.sample(g.row_ptr, g.col, v, 5, 0, 64)
    b = oracle.sample_threads(g.row_ptr, g.col, v, 5, 0, 64, threads=4)
    assert np.array_equal(a.cnt1, b.cnt1) and np.array_equal(a.cnt2, b.cnt2)
    assert a.sum_y1 == b.sum_y1 and a.sum_y2 == b.sum_y2


# ------------------------------------------------ Kirchhoff index, random-walk betweenness (Section 5)

def test_kirchhoff_index_closed_forms():
    """Tr(L^+) of K_n is (n-1)/n (L^+ = (I - J/n)/n); of the path P_n it is
    (n^2 - 1)/6 (the sum of resistances over node pairs, (n^3 - n)/6, is
    n Tr(L^+)); of the cycle C_n it is (n^2 - 1)/12."""
    import oracle.dense as D
    for n in (3, 5, 9):
        g = I.complete(n)
        assert D.kirchhoff(n, g.row_ptr, g.col) == pytest.approx((n - 1) / n, rel=1e-12)
        g = I.path(n)
        assert D.kirchhoff(n, g.row_ptr, g.col) == pytest.approx((n * n - 1) / 6.0, rel=1e-12)
        g = I.cycle(n)
        assert D.kirchhoff(n, g.row_ptr, g.col) == pytest.approx((n * n - 1) / 12.0, rel=1e-12)


def test_rw_betweenness_closed_form_and_ldiag_route():
    """On K_n every node has c_b = 1/n + 1/(2(n-1)); from_ldiag on the dense
    diagonal reproduces the dense definition on an irregular graph."""
    import oracle.dense as D
    n = 7
    g = I.complete(n)
    np.testing.assert_allclose(D.rw_betweenness(n, g.row_ptr, g.col), 1.0 / n + 1.0 / (2 * (n - 1)), rtol=1e-12)
    g = I.ba(60, 2, seed=3)
    lp = np.diag(D.pinv_laplacian(g.n, g.row_ptr, g.col))
    tr, cb = D.from_ldiag(lp)
    assert tr == pytest.approx(float(lp.sum()), rel=1e-13)
    assert np.all(cb > 1.0 / g.n) and np.argmax(cb) == np.argmin(lp)


@pytest.mark.parametrize("paths", [False, True], ids=["own_draws", "stack_paths"])
def test_fixed_start_passes_estimate_a_row_of_lv_inverse(paths):
    """Section 4.2 lemmas ("v-absorbed walk", "loop-erased walk"): the passes
    of u on a v-absorbed walk from s -- or on the loop-included path from s
    of a Wilson run's stacks -- have mean d_u (L_v^{-1})_{su}.  With the first
    absorbed walk started at a fixed s, cnt2 / (omega d) matches row s of the
    dense L_v^{-1} within 6 standard errors at every node (batch means), and
    the pass at s itself is counted (the row's diagonal entry is >= 1 / d_s)."""
    g = I.ba(80, 2, seed=9)
    v = oracle.root_max_degree(g.row_ptr)
    d = np.diff(g.row_ptr).astype(np.float64)
    lv = D.lv_inverse(g.n, g.row_ptr, g.col, v)
    for s in (int(np.argmin(d)), (v + 1) % g.n):
        if s == v:
            continue
        rows = []
        for b in range(20):
            c = oracle.sample_threads(g.row_ptr, g.col, v, 31, 400 * b, 400, 4, paths=paths, path_start=s)
            rows.append(c.cnt2.astype(np.float64) / (400 * d))
        rows = np.array(rows)
        mean, se = rows.mean(axis=0), rows.std(axis=0, ddof=1) / np.sqrt(len(rows))
        keep = np.arange(g.n) != v
        assert np.all(np.abs(mean - lv[s])[keep] <= 6 * se[keep] + 1e-12), np.max(np.abs(mean - lv[s]) / (se + 1e-300))
        assert np.all(rows[:, s] >= 1.0 / d[s] - 1e-15)
        assert np.all(rows[:, v] == 0.0)
