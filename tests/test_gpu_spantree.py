"""GPU parity of the SpanTree estimators (Alg. 1, Alg. 3) with the oracle
(oracle/spantree.py): the integer flow sums bit-exact for the same trees
(same Philox keying as lap_sample), FP64 estimates within 1e-12, split calls
equal to one call, and the estimates consistent with the dense values."""
import numpy as np
import pytest

import oracle.dense as D
import oracle.spantree as S
from paper_2311_10290_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2311_10290_gb300.lap import LapGraph  # noqa: E402


def run(g, root, seed, splits, ws=1 << 27):
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=ws)
    try:
        v = G.set_root(root)
        for c in splits:
            G.spantree_sample(c, seed)
        x1, x2, x2d, om = G.spantree_sums()
        ld, ec, kc = G.spantree_estimates()
    finally:
        G.close()
    return v, x1, x2, x2d, om, ld, ec, kc


@pytest.mark.parametrize("name,maker,root", [
    ("ba", lambda: I.ba(800, 3, seed=2), -1),
    ("er", lambda: I.er(400, 0.02, seed=3), -1),
    ("rmat", lambda: I.rmat(9, 6, seed=4), -1),
    ("path_end", lambda: I.path(70), 0),
    ("star_leaf", lambda: I.star(50), 3),
    ("k4e", lambda: I.k4_minus_edge(), 0),
], ids=["ba", "er", "rmat", "path_end", "star_leaf", "k4e"])
def test_spantree_sums_bit_exact(name, maker, root):
    g = maker()
    k, seed = 48, 19
    v, x1, x2, x2d, om, ld, ec, kc = run(g, root, seed, [20, 28])
    assert om == k
    X1, X2, X2d = S.spantree_sample(g.row_ptr, g.col, v, seed, 0, k)
    assert np.array_equal(x1, X1) and np.array_equal(x2, X2) and np.array_equal(x2d, X2d)
    ldo, eco, kco = S.spantree_estimates(g.row_ptr, v, k, X1, X2, X2d)
    d = np.diff(g.row_ptr).astype(np.float64)
    scale = np.abs(X1) / k + 2.0 * np.abs(X2) / (g.n * k) + abs(ldo[v])
    assert np.all(np.abs(ld - ldo) <= 1e-12 * scale + 1e-300)
    np.testing.assert_allclose(ec, eco, rtol=1e-11)
    kscale = (float(d @ np.abs(X1)) + float(d @ np.abs(X2d)) / g.row_ptr[-1]) / k
    assert abs(kc - kco) <= 1e-12 * kscale


def test_small_workspace_many_chunks_equal_one_run():
    """Trees in flight limited to 3 by the workspace: the sums are those of
    one run over all ids."""
    g = I.ba(600, 2, seed=7)
    a = run(g, -1, 5, [40], ws=8 * g.n * 3)
    b = run(g, -1, 5, [13, 27], ws=1 << 26)
    for x, y in zip(a[1:4], b[1:4]):
        assert np.array_equal(x, y)


def test_spantree_estimates_near_dense():
    """The estimators are unbiased (Section 4.1, Section 5.1): over 30 GPU
    batches of 100 trees, every node's mean (L^+)_uu and the mean Kemeny
    estimate lie within 6 standard errors of the batch means (Student t with
    29 degrees of freedom: P(|t| > 6) is about 1.4e-6 per node, so about
    4e-4 for the whole graph) of the dense FP64 values."""
    g = I.er(300, 0.03, seed=6)
    batches, per = 30, 100
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 28)
    lds, kcs = [], []
    try:
        v = G.set_root(-1)
        prev = [np.zeros(g.n, dtype=np.int64)] * 3
        for b in range(batches):
            G.spantree_sample(per, 9)
            x1, x2, x2d, om = G.spantree_sums()
            cur = [x1.astype(np.int64), x2.astype(np.int64), x2d.astype(np.int64)]
            d1, d2, d2d = (c - q for c, q in zip(cur, prev))
            prev = cur
            ld, _, kc = S.spantree_estimates(g.row_ptr, v, per, d1, d2, d2d)
            lds.append(ld)
            kcs.append(kc)
    finally:
        G.close()
    lds, kcs = np.array(lds), np.array(kcs)
    exact = np.diag(D.pinv_laplacian(g.n, g.row_ptr, g.col))
    se = lds.std(axis=0, ddof=1) / np.sqrt(batches)
    z = np.abs(lds.mean(axis=0) - exact) / se
    assert np.all(z < 6.0), (np.max(z), int(np.argmax(z)))
    kse = kcs.std(ddof=1) / np.sqrt(batches)
    assert abs(kcs.mean() - D.kemeny(g.n, g.row_ptr, g.col)) < 6.0 * kse


def test_spantree_and_lewalk_share_the_trees():
    """Tree i of lap_spantree_sample is the tree of lap_sample's sample id i:
    the oracle's trees for those ids give the GPU sums (checked above), and
    both estimators of the same handle run side by side."""
    g = I.ba(500, 3, seed=1)
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 26)
    try:
        G.set_root()
        G.sample(200, 3)
        e1 = G.ecc()
        G.spantree_sample(30, 3)
        G.sample(100, 3)                    # the LEWalk path reuses the workspace afterwards
        c1, _, s = G.counts()
        _, _, _, om = G.spantree_sums()
    finally:
        G.close()
    assert int(s[0]) == 300 and om == 30
    c = __import__("oracle").sample(g.row_ptr, g.col, int(np.argmax(np.diff(g.row_ptr))), 3, 0, 300,
                                    keep_per_sample=False)
    assert np.array_equal(c1, c.cnt1)
    assert np.all(np.isfinite(e1))
