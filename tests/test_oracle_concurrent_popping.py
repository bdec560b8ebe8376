"""Order independence of Wilson's algorithm under concurrent walkers (the
stack representation of Fig. 1: every draw at a node is the next entry of
that node's stack), pinned against the sequential oracle: several walkers share one sample's Wilson run, each following and
drawing the tops of the nodes' stacks (draw j of node u in sample i is the
Philox counter (u, j, i, 0)), under this protocol:

- a walker at its head u takes u's pending arrow if an aborted walker left
  one there, else draws u's next stack entry (a visit of u);
- landing on the tree commits the walker's path; landing on its own path
  pops the closed cycle (those nodes' arrows are consumed: the next visit
  draws afresh);
- landing on another walker's path: a lower-numbered walker waits and tries
  the same arrow again later; a higher-numbered one aborts, leaving every
  arrow of its path pending on its nodes, and starts elsewhere.

Only genuine cycles of stack tops are ever popped, so by the stack theorem
the popped cycles, hence the draws per node (visits) and the final tree, are
those of the sequential run whatever the interleaving.  The simulation runs
random interleavings and compares with oracle.sample (cnt1 = visits per node,
the tree).  This is the correctness argument for sampling one Wilson run with
several GPU lanes, checked before any such kernel exists."""
import numpy as np
import pytest

import oracle
from paper_2311_10290_gb300 import inputs as I


class Stacks:
    """Draw j of node u in sample i, as the samplers key it."""

    def __init__(self, g, seed, i):
        self.rp, self.col, self.seed, self.i = g.row_ptr, g.col, seed, i
        self.cache = {}

    def __call__(self, u, j):
        key = (u, j)
        if key not in self.cache:
            blk = oracle.philox_block([u, j, self.i, 0], [self.seed & 0xFFFFFFFF, self.seed >> 32])
            r = int(blk[0]) | (int(blk[1]) << 32)
            deg = int(self.rp[u + 1] - self.rp[u])
            self.cache[key] = int(self.col[int(self.rp[u]) + ((r * deg) >> 64)])
        return self.cache[key]


def concurrent_wilson(g, v, seed, i, walkers, rng, keep_pending=True, max_rounds=10 ** 6):
    n = g.n
    draw = Stacks(g, seed, i)
    k = [0] * n                  # draws taken at each node (= visits)
    pending = [-1] * n           # an aborted walker's arrow left on a free node
    arrow = [-1] * n             # the arrow a path (or, at the end, the tree) follows out of a node
    owner = [-1] * n
    intree = [False] * n
    intree[v] = True
    paths = [[] for _ in range(walkers)]
    left = n - 1
    for _ in range(max_rounds):
        if left == 0:
            return k, arrow
        for wk in rng.permutation(walkers):
            wk = int(wk)
            path = paths[wk]
            if not path:
                free = [u for u in range(n) if not intree[u] and owner[u] < 0]
                if free:
                    s = free[int(rng.integers(len(free)))] if rng.random() < 0.5 else free[0]
                    owner[s] = wk
                    path.append(s)
                continue
            u = path[-1]
            if arrow[u] < 0:
                if pending[u] >= 0:
                    arrow[u], pending[u] = pending[u], -1
                else:
                    arrow[u] = draw(u, k[u])
                    k[u] += 1
            w = arrow[u]
            if intree[w]:
                for x in path:
                    intree[x] = True
                    owner[x] = -1
                left -= len(path)
                path.clear()
            elif owner[w] == wk:
                while path[-1] != w:
                    x = path.pop()
                    owner[x] = -1
                    arrow[x] = -1
                arrow[w] = -1
            elif owner[w] >= 0:
                if wk > owner[w]:
                    for x in path:
                        owner[x] = -1
                        pending[x], arrow[x] = (arrow[x] if keep_pending else -1), -1
                    path.clear()
                # else: wait, and try the same arrow again next round
            else:
                owner[w] = wk
                path.append(w)
    raise AssertionError("no progress within %d rounds" % max_rounds)


CASES = [
    ("k4e", I.k4_minus_edge, 0),
    ("ba60", lambda: I.ba(60, 2, seed=4), -1),
    ("er80", lambda: I.er(80, 0.08, seed=6), -1),
    ("cycle30", lambda: I.cycle(30), 0),
    ("star20_leaf", lambda: I.star(20), 5),
    ("path25_end", lambda: I.path(25), 0),
]


@pytest.mark.parametrize("walkers", [2, 4, 8])
@pytest.mark.parametrize("name,maker,root", CASES, ids=[c[0] for c in CASES])
def test_concurrent_walkers_give_the_sequential_counts_and_tree(name, maker, root, walkers):
    g = maker()
    v = oracle.root_max_degree(g.row_ptr) if root < 0 else root
    seed = 0xC0FFEE + walkers
    rng = np.random.default_rng(len(name) * 31 + walkers)
    for i in range(4):
        k, arrow = concurrent_wilson(g, v, seed, i, walkers, rng)
        ref = oracle.sample(g.row_ptr, g.col, v, seed, i, 1, keep_tree=True)
        assert [int(x) for x in ref.cnt1] == k
        tree = [int(x) for x in ref.tree[0]]
        assert all(arrow[u] == tree[u] for u in range(g.n) if u != v)


def test_dropping_the_aborted_arrows_breaks_the_counts():
    """The pending arrows are what keeps an abort exact: a walker that gives
    up its path while its drawn arrows are forgotten (the next visitor draws
    again) pops stack entries that are not on any cycle, so the counts move
    away from the sequential run."""
    g = I.ba(60, 2, seed=4)
    v = oracle.root_max_degree(g.row_ptr)
    differ = 0
    for i in range(8):
        k, _ = concurrent_wilson(g, v, 123, i, 4, np.random.default_rng(i), keep_pending=False)
        ref = oracle.sample(g.row_ptr, g.col, v, 123, i, 1)
        differ += [int(x) for x in ref.cnt1] != k
    assert differ >= 4


@pytest.fixture(scope="module")
def threaded(tmp_path_factory):
    """tests/concurrent_popping.c built with gcc (pthreads, C11 atomics)."""
    import ctypes
    import os
    import subprocess
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "concurrent_popping.c")
    lib = str(tmp_path_factory.mktemp("popping") / "libpopping.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-pthread", "-fPIC", "-shared", "-o", lib, src])
    so = ctypes.CDLL(lib)
    p = ctypes.c_void_p
    so.concurrent_popping.restype = ctypes.c_int
    so.concurrent_popping.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, p, ctypes.c_int32,
                                      ctypes.c_uint64, ctypes.c_long, p, p]
    return so


# Larger graphs keep several threads inside one sample at once (aborts, waits
# and lost claims all occur on these).
THREAD_CASES = CASES + [
    ("ba2000", lambda: I.ba(2000, 3, seed=1), -1),
    ("er1000", I.er_1000, -1),
]


@pytest.mark.parametrize("walkers", [2, 4, 16])
@pytest.mark.parametrize("name,maker,root", THREAD_CASES, ids=[c[0] for c in THREAD_CASES])
def test_threads_sharing_one_sample_give_the_sequential_counts_and_tree(threaded, name, maker, root, walkers):
    """The same protocol on real threads: one 64-bit word per node changed by
    compare-and-swap (claiming a free node is the only contended write), the
    draws given as a table in the oracle's keying.  Every run, whatever the
    scheduling, ends with the sequential oracle's visits per node and tree."""
    g = maker()
    v = oracle.root_max_degree(g.row_ptr) if root < 0 else root
    seed = 0xBEEF + walkers
    for i in range(3):
        ref = oracle.sample(g.row_ptr, g.col, v, seed, i, 1, keep_tree=True)
        kmax = int(ref.cnt1.max()) + 1
        draw = Stacks(g, seed, i)
        table = np.array([[draw(u, j) for j in range(kmax)] for u in range(g.n)], dtype=np.int32)
        for rep in range(3):
            k = np.zeros(g.n, dtype=np.int32)
            arrow = np.zeros(g.n, dtype=np.int32)
            rc = threaded.concurrent_popping(g.n, v, kmax, table.ctypes.data, walkers, 1000 * i + rep, 10 ** 7,
                                             k.ctypes.data, arrow.ctypes.data)
            assert rc == 0, rc
            assert np.array_equal(k, ref.cnt1.astype(np.int32))
            tree = np.array(ref.tree[0], dtype=np.int32)
            assert np.array_equal(arrow, tree)
