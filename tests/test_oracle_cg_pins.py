"""Pins for the sparse solves of the large-graph ground truth (oracle/cg.py):
closed forms on a path rooted at one end, the dense inverse of L_v on small
graphs, and L^+_vv / E[Y2] against the dense pseudo-inverse.  CPU only."""
import numpy as np
import pytest

import oracle.cg as CG
import oracle.dense as D
from paper_2311_10290_gb300 import inputs as I


def test_path_rooted_at_an_end_closed_forms():
    """On the path 0 - 1 - ... - (n-1) grounded at 0, (L_0^{-1})_jk = min(j, k)
    (the resistance shared by the paths from j and k to 0), so
    (L_0^{-1} 1)_j = j (j + 1) / 2 + j (n - 1 - j), and the hitting time of 0
    from j is j (2 (n - 1) - j)."""
    n = 40
    g = I.path(n)
    j = np.arange(n, dtype=np.float64)
    x, it, res = CG.solve_lv(g.row_ptr, g.col, 0, np.ones(n))
    np.testing.assert_allclose(x, j * (j + 1) / 2 + j * (n - 1 - j), rtol=1e-10)
    p = CG.exact_parts(g.row_ptr, g.col, 0)
    np.testing.assert_allclose(p["hitting"], j * (2 * (n - 1) - j), rtol=1e-10)
    assert res <= 1e-12


@pytest.mark.parametrize("g", [I.k4_minus_edge(), I.er(120, 0.05, seed=2), I.ba(300, 2, seed=3),
                               I.rmat(8, 6, seed=4)], ids=["k4e", "er", "ba", "rmat"])
def test_solves_equal_the_dense_inverse(g):
    v = int(np.argmax(np.diff(g.row_ptr)))
    li = D.lv_inverse(g.n, g.row_ptr, g.col, v)
    rng = np.random.default_rng(1)
    for b in (np.ones(g.n), np.diff(g.row_ptr).astype(np.float64), rng.standard_normal(g.n)):
        x, _, _ = CG.solve_lv(g.row_ptr, g.col, v, b)
        want = li @ np.where(np.arange(g.n) == v, 0.0, b)
        np.testing.assert_allclose(x, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())
        assert x[v] == 0.0


@pytest.mark.parametrize("g", [I.er(150, 0.04, seed=5), I.ba(400, 3, seed=6)], ids=["er", "ba"])
def test_exact_parts_match_the_pseudo_inverse(g):
    """L^+_vv = (1/n^2) 1^T L_v^{-1} 1 (Section 3.1) and E[Y2] =
    (1/2m) d^T L_v^{-1} d (Alg. 4) against the dense pseudo-inverse and the
    dense expectation; y2 against the dense row sums."""
    v = int(np.argmax(np.diff(g.row_ptr)))
    p = CG.exact_parts(g.row_ptr, g.col, v)
    pinv = D.pinv_laplacian(g.n, g.row_ptr, g.col)
    assert p["lvv"] == pytest.approx(pinv[v, v], rel=1e-9)
    e = D.expectations(g.n, g.row_ptr, g.col, v)
    assert p["ey2"] == pytest.approx(e["y2"], rel=1e-9)
    d = np.diff(g.row_ptr).astype(np.float64)
    np.testing.assert_allclose(p["y2"] * d, e["passes"], rtol=1e-9, atol=1e-12)
