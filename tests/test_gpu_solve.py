"""GPU FP64 solves with L_v (lap_lv_solve) against the oracle's sparse solver
(oracle/cg.py, itself pinned by closed forms and the dense inverse): the two
run the same preconditioned conjugate-gradient method in different
summation orders and stop at relative residual 1e-12, so the solutions
agree to 1e-9 relative."""
import numpy as np
import pytest

import oracle.cg as CG
from paper_2311_10290_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2311_10290_gb300.lap import LapGraph  # noqa: E402


@pytest.mark.parametrize("maker,root", [(lambda: I.path(60), 0), (lambda: I.er(500, 0.02, seed=3), -1),
                                        (lambda: I.ba(4000, 3, seed=4), -1), (lambda: I.rmat(12, 8, seed=5), -1)],
                         ids=["path_end", "er", "ba", "rmat"])
def test_lv_solve_matches_oracle(maker, root):
    g = maker()
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 22)
    try:
        v = G.set_root(root)
        d = np.diff(g.row_ptr).astype(np.float64)
        for b in (np.ones(g.n), d, np.random.default_rng(1).standard_normal(g.n)):
            x, it, res = G.lv_solve(b)
            xd, _, _ = G.lv_solve(torch.from_numpy(b).cuda())
            want, _, _ = CG.solve_lv(g.row_ptr, g.col, v, b)
            assert res <= 1e-12 and it > 0
            np.testing.assert_allclose(x, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())
            assert np.array_equal(x, xd.cpu().numpy())        # host and device paths: the same iterates
            assert x[v] == 0.0
    finally:
        G.close()


def test_lv_solve_full_size_ba():
    """The 10^6-node Barabasi-Albert workload graph: L_v^{-1} 1 and L_v^{-1} d."""
    g = I.ba_1m()
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 26)
    try:
        v = G.set_root()
        d = np.diff(g.row_ptr).astype(np.float64)
        for b in (np.ones(g.n), d):
            x, it, res = G.lv_solve(b)
            want, _, _ = CG.solve_lv(g.row_ptr, g.col, v, b)
            np.testing.assert_allclose(x, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())
    finally:
        G.close()
