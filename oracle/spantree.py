"""Oracle for the SpanTree estimators: Alg. 1 (ECC) and Alg. 3 (Kemeny's constant).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): plain numpy and Python
loops, exact integers.

Section 4.1: the electrical flow of G is the average of the flows sent on
its uniform spanning trees, so a voltage of G (the sum of edge flows along
any fixed path to the landmark v) is the average over trees of the same sum
of tree flows.  With a fixed BFS tree from v giving the path P_BFS[u], a
sampled spanning tree T (parent array next[], rooted at v) contributes, per
node u and per edge (e1 -> e2) of P_BFS[u] (e2 the BFS parent of e1):

  x1(u): the flow of one unit from u to v on T is 1 on the tree path from u:
         +1 if next[e1] == e2 and e1 is on T's path from u (u in subtree(e1)),
         -1 if next[e2] == e1 and e2 is on T's path from u (u in subtree(e2));
         E[x1(u)] = (L_v^{-1})_uu                                   (Alg. 1)
  x2(u): 1/n injected at every node: the tree edge (a, next[a]) carries
         |subtree(a)| / n, whatever u is:
         +|subtree(e1)| if next[e1] == e2,  -|subtree(e2)| if next[e2] == e1,
         scaled by 1/n;  E[x2(u)] = (1/n) e_u^T L_v^{-1} 1            (Alg. 1)
  x2d(u): d_w / 2m injected at every w: edge (a, next[a]) carries
         (sum of d_w over subtree(a)) / 2m;  then
         E[sum_u d_u x1(u)] = Tr((I - P_v)^{-1}) and
         E[sum_u d_u x2d(u)] = (1/2m) d^T L_v^{-1} d                 (Alg. 3)

Readings (the printed pseudocode is garbled in two places): the ancestor
test is "e1 is an ancestor of u" (u's DFS interval inside e1's), as the text
states, not the printed inclusion the other way; and the x2 terms take every
tree edge of P_BFS[u] (the tree flow of the all-node injection does not depend
on u), not only those on u's tree path.  The BFS parent of u is its
smallest-id neighbour one hop closer to v.

Sums are kept as exact integers per node (x1, |subtree| sums, degree sums);
the estimates divide once at the end.
"""
from __future__ import annotations

import math

import numpy as np


def bfs_parent(row_ptr, col, v):
    """Parent of every node in the BFS tree from v: the smallest-id
    neighbour with hop distance one less (-1 at v)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    cl = np.asarray(col, dtype=np.int64)
    n = rp.size - 1
    hops = np.full(n, -1, dtype=np.int64)
    hops[v] = 0
    frontier = [int(v)]
    while frontier:
        nxt = []
        for u in frontier:
            for w in cl[rp[u]:rp[u + 1]]:
                if hops[w] < 0:
                    hops[w] = hops[u] + 1
                    nxt.append(int(w))
        frontier = nxt
    par = np.full(n, -1, dtype=np.int64)
    for u in range(n):
        if u == v:
            continue
        cand = [int(w) for w in cl[rp[u]:rp[u + 1]] if hops[w] == hops[u] - 1]
        par[u] = min(cand)
    return par


def tree_intervals(parent, v, deg):
    """Preorder index, subtree node count and subtree degree sum of every
    node of the tree given by parent[] (rooted at v), by an iterative DFS."""
    n = len(parent)
    children = [[] for _ in range(n)]
    for u in range(n):
        if u != v:
            children[int(parent[u])].append(u)
    pre = np.zeros(n, dtype=np.int64)
    size = np.ones(n, dtype=np.int64)
    dsum = np.asarray(deg, dtype=np.int64).copy()
    order = []
    stack = [int(v)]
    while stack:
        u = stack.pop()
        pre[u] = len(order)
        order.append(u)
        stack.extend(reversed(children[u]))
    for u in reversed(order):
        if u != v:
            size[int(parent[u])] += size[u]
            dsum[int(parent[u])] += dsum[u]
    return pre, size, dsum


def tree_terms(row_ptr, col, v, bpar, parent):
    """Per-node integer terms of one spanning tree: (x1, x2 * n, x2d * 2m)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    n = rp.size - 1
    deg = rp[1:] - rp[:-1]
    pre, size, dsum = tree_intervals(parent, v, deg)

    def inside(u, a):          # u in subtree(a), i.e. a on T's path from u to v
        return pre[a] <= pre[u] < pre[a] + size[a]

    x1 = np.zeros(n, dtype=np.int64)
    x2 = np.zeros(n, dtype=np.int64)
    x2d = np.zeros(n, dtype=np.int64)
    for u in range(n):
        e1 = u
        while e1 != v:
            e2 = int(bpar[e1])
            if int(parent[e1]) == e2:
                x2[u] += size[e1]
                x2d[u] += dsum[e1]
                if inside(u, e1):
                    x1[u] += 1
            elif e2 != v and int(parent[e2]) == e1:
                x2[u] -= size[e2]
                x2d[u] -= dsum[e2]
                if inside(u, e2):
                    x1[u] -= 1
            e1 = e2
    return x1, x2, x2d


def spantree_sums(row_ptr, col, v, trees):
    """Sums over the given trees (parent arrays, -1 at v) of the per-node terms."""
    bpar = bfs_parent(row_ptr, col, v)
    n = len(row_ptr) - 1
    X1 = np.zeros(n, dtype=np.int64)
    X2 = np.zeros(n, dtype=np.int64)
    X2d = np.zeros(n, dtype=np.int64)
    for t in trees:
        a, b, c = tree_terms(row_ptr, col, v, bpar, t)
        X1 += a
        X2 += b
        X2d += c
    return X1, X2, X2d


def spantree_sample(row_ptr, col, v, seed, first, count):
    """Alg. 1 / Alg. 3 sums over the Wilson trees of sample ids
    [first, first+count) (the LEWalk oracle's trees, same Philox keying)."""
    import oracle
    c = oracle.sample(row_ptr, col, v, seed, first, count, keep_per_sample=False, keep_tree=True)
    return spantree_sums(row_ptr, col, v, c.tree)


def spantree_estimates(row_ptr, v, omega, X1, X2, X2d):
    """Returns (ldiag, ecc, kemeny) from the integer sums (FP64, compensated sums)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    n = rp.size - 1
    deg = (rp[1:] - rp[:-1]).astype(np.float64)
    two_m = float(rp[-1])
    w = float(omega)
    x1 = np.asarray(X1, dtype=np.float64) / w
    x2 = np.asarray(X2, dtype=np.float64) / (n * w)
    mean_x2 = math.fsum(x2.tolist()) / n
    ld = x1 - 2.0 * x2 + mean_x2
    ld[v] = mean_x2
    tr = math.fsum(ld.tolist())
    ecc = (n - 1) / (n * ld + tr)
    t1 = math.fsum((deg * np.asarray(X1, dtype=np.float64)).tolist()) / w
    t2 = math.fsum((deg * np.asarray(X2d, dtype=np.float64)).tolist()) / (two_m * w)
    return ld, ecc, t1 - t2
