"""Pins of the SpanTree oracle (oracle/spantree.py; Alg. 1 and Alg. 3).

Averaged over ALL spanning trees (enumerated by brute force), the per-tree
terms must give the exact values (dense FP64): (L_v^{-1})_uu, (1/n) e_u^T
L_v^{-1} 1, Tr((I - P_v)^{-1}), (1/2m) d^T L_v^{-1} d, and so L^+_uu, ECC and
Kemeny's constant.  The paper's worked example K4-e with 8 trees gives
(L^+)_vv = 5/16.  The containment test as printed in Alg. 1 (the other way
round) is shown to be biased, which fixes the reading."""
import itertools

import numpy as np
import pytest
from _golden import read_kv

import oracle.dense as D
import oracle.spantree as S
from paper_2311_10290_gb300 import inputs as I


def all_trees_rooted(g, v):
    """Every spanning tree of g as a parent array rooted at v (brute force)."""
    edges = [(u, int(w)) for u in range(g.n) for w in g.col[g.row_ptr[u]:g.row_ptr[u + 1]] if u < w]
    out = []
    for sub in itertools.combinations(edges, g.n - 1):
        adj = [[] for _ in range(g.n)]
        for a, b in sub:
            adj[a].append(b)
            adj[b].append(a)
        par = [-2] * g.n
        par[v] = -1
        stack = [v]
        while stack:
            u = stack.pop()
            for w in adj[u]:
                if par[w] == -2:
                    par[w] = u
                    stack.append(w)
        if all(p != -2 for p in par):
            out.append(np.array(par, dtype=np.int64))
    return out


def small_graphs():
    yield "k4e", I.k4_minus_edge()
    yield "k4", I.complete(4)
    yield "c5", I.cycle(5)
    yield "p5", I.path(5)
    yield "star5", I.star(5)
    g = I.er(7, 0.55, seed=11)
    yield "er7", g


@pytest.mark.parametrize("name,g", list(small_graphs()), ids=[x for x, _ in small_graphs()])
def test_average_over_all_trees_is_exact(name, g):
    deg = np.diff(g.row_ptr).astype(np.float64)
    for v in sorted({0, g.n - 1, int(np.argmax(deg))}):
        trees = all_trees_rooted(g, v)
        T = len(trees)
        X1, X2, X2d = S.spantree_sums(g.row_ptr, g.col, v, trees)
        lv = D.lv_inverse(g.n, g.row_ptr, g.col, v)
        np.testing.assert_allclose(X1 / T, np.diag(lv), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(X2 / (g.n * T), lv.sum(axis=1) / g.n, rtol=1e-12, atol=1e-12)
        assert float(deg @ X1) / T == pytest.approx(float(deg @ np.diag(lv)), rel=1e-12)
        two_m = float(g.row_ptr[-1])
        assert float(deg @ X2d) / (two_m * T) == pytest.approx(float(deg @ lv @ deg) / two_m, rel=1e-12)
        ld, ec, kc = S.spantree_estimates(g.row_ptr, v, T, X1, X2, X2d)
        np.testing.assert_allclose(ld, np.diag(D.pinv_laplacian(g.n, g.row_ptr, g.col)), rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(ec, D.ecc(g.n, g.row_ptr, g.col), rtol=1e-11)
        assert kc == pytest.approx(D.kemeny(g.n, g.row_ptr, g.col), rel=1e-11)


def test_worked_example_k4e():
    """Section 4.1: over the 8 spanning trees of K4-e, the flows give (L^+)_vv = 5/16."""
    kv = read_kv("k4e_worked_example.txt")
    g = I.k4_minus_edge()
    trees = all_trees_rooted(g, 0)
    assert len(trees) == int(kv["spanning_trees"])
    X1, X2, X2d = S.spantree_sums(g.row_ptr, g.col, 0, trees)
    ld, _, _ = S.spantree_estimates(g.row_ptr, 0, len(trees), X1, X2, X2d)
    assert ld[0] == pytest.approx(float(kv["ldag_vv"]), rel=1e-13)


def test_printed_containment_direction_is_biased():
    """With the inclusion of Alg. 1 taken literally (e1's interval inside u's),
    the x1 average over all trees of K4-e misses (L_v^{-1})_uu; the reading
    used (u's interval inside e1's, 'e1 is an ancestor of u') is exact."""
    g = I.k4_minus_edge()
    v = 0
    trees = all_trees_rooted(g, v)
    bpar = S.bfs_parent(g.row_ptr, g.col, v)
    deg = np.diff(g.row_ptr)
    lit = np.zeros(g.n)
    for t in trees:
        pre, size, _ = S.tree_intervals(t, v, deg)
        for u in range(g.n):
            e1 = u
            while e1 != v:
                e2 = int(bpar[e1])
                if t[e1] == e2 and pre[u] <= pre[e1] < pre[u] + size[u]:
                    lit[u] += 1
                elif e2 != v and t[e2] == e1 and pre[u] <= pre[e2] < pre[u] + size[u]:
                    lit[u] -= 1
                e1 = e2
    lv = np.diag(D.lv_inverse(g.n, g.row_ptr, g.col, v))
    assert np.max(np.abs(lit / len(trees) - lv)) > 0.05


def test_bfs_parent_is_one_hop_closer_and_smallest():
    g = I.ba(200, 3, seed=5)
    v = 0
    par = S.bfs_parent(g.row_ptr, g.col, v)
    hops = D_hops(g, v)
    for u in range(g.n):
        if u == v:
            assert par[u] == -1
            continue
        nb = g.col[g.row_ptr[u]:g.row_ptr[u + 1]]
        closer = [int(w) for w in nb if hops[w] == hops[u] - 1]
        assert par[u] == min(closer)


def D_hops(g, v):
    import oracle.cv as CV
    return CV.bfs_hops(g.row_ptr, g.col, v)


def test_sampled_trees_estimate_within_error():
    """Wilson trees of the LEWalk oracle (same Philox keying as the GPU):
    SpanTree estimates of Tr((I-P_v)^{-1}) - (1/2m) d^T L_v^{-1} d = kappa
    and of L^+_uu fall within 6 standard errors of the dense values."""
    g = I.ba(60, 2, seed=8)
    v = int(np.argmax(np.diff(g.row_ptr)))
    k = 400
    import oracle
    c = oracle.sample(g.row_ptr, g.col, v, 5, 0, k, keep_per_sample=False, keep_tree=True)
    bpar = S.bfs_parent(g.row_ptr, g.col, v)
    deg = np.diff(g.row_ptr).astype(np.float64)
    per = np.array([float(deg @ a) - float(deg @ c2) / g.row_ptr[-1]
                    for a, _, c2 in (S.tree_terms(g.row_ptr, g.col, v, bpar, t) for t in c.tree)])
    kc = D.kemeny(g.n, g.row_ptr, g.col)
    assert abs(per.mean() - kc) < 6 * per.std() / np.sqrt(k) + 1e-12
    X1, X2, X2d = S.spantree_sums(g.row_ptr, g.col, v, c.tree)
    ld, _, kc_est = S.spantree_estimates(g.row_ptr, v, k, X1, X2, X2d)
    assert kc_est == pytest.approx(per.mean(), rel=1e-12)
    exact = np.diag(D.pinv_laplacian(g.n, g.row_ptr, g.col))
    assert np.mean(np.abs(ld - exact) / exact) < 0.1
