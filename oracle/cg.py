"""Sparse FP64 solves with L_v for graphs too large for the dense estimand.

TEST INFRASTRUCTURE ONLY: imported by the test suite and the benchmark's
accuracy measurement (the exact parts of the ground truth on the large
graphs), never by the library.

``L_v`` is the Laplacian ``L = D - A`` without row and column ``v``
(Section 3.1).  Two of the quantities the samplers estimate are linear in
``L_v^{-1}`` applied to a known vector, so one solve each gives them exactly
(to the solver's tolerance):

* ``r = L_v^{-1} 1``: the uniform-start walks' target, ``y2(u) = r_u / n``
  (Alg. 2; the lemma of Section 4.2 on the passes of a v-absorbed walk), and
  with it ``(L^+)_vv = (1/n^2) 1^T r`` and the row-sum terms of every
  ``(L^+)_uu`` (Section 3.1, element-wise Theorem 1);
* ``h = L_v^{-1} d``: the hitting times ``h(u, v)`` (Section 3.2), and
  ``E[Y2] = (1/2m) d^T h``, the term Alg. 4 subtracts from ``Tr((I-P_v)^{-1})``
  to give Kemeny's constant (Section 5).

The solver is the conjugate-gradient method (Hestenes and Stiefel, 1952) with
the Jacobi preconditioner ``D^{-1}`` (``L_v`` is symmetric positive definite
for a connected graph), written out step by step; the matrix-vector product
is scipy's CSR product.
"""
from __future__ import annotations

import numpy as np


def _lv_operator(row_ptr, col, v):
    """(matvec over the n-1 non-root nodes, their degrees, index map)."""
    import scipy.sparse as sp
    rp = np.asarray(row_ptr, dtype=np.int64)
    cl = np.asarray(col, dtype=np.int64)
    n = rp.size - 1
    d = (rp[1:] - rp[:-1]).astype(np.float64)
    A = sp.csr_matrix((np.ones(cl.size), cl, rp), shape=(n, n))
    keep = np.arange(n) != v
    idx = np.nonzero(keep)[0]
    Lv = (sp.diags(d) - A)[idx][:, idx].tocsr()
    return (lambda x: Lv @ x), d[idx], idx


def solve_lv(row_ptr, col, v, b, rtol=1e-12, maxiter=100000):
    """x = L_v^{-1} b for a length-n right-hand side b (b[v] ignored); returns
    (x with x[v] = 0, iterations, final relative residual ||b - L_v x|| / ||b||)."""
    n = np.asarray(row_ptr).size - 1
    matvec, dv, idx = _lv_operator(row_ptr, col, v)
    rhs = np.asarray(b, dtype=np.float64)[idx]
    bnorm = float(np.linalg.norm(rhs))
    x = np.zeros(idx.size)
    if bnorm == 0.0:
        return np.zeros(n), 0, 0.0
    r = rhs.copy()                 # residual b - L_v x for x = 0
    z = r / dv                     # preconditioned residual
    p = z.copy()
    rz = float(r @ z)
    it = 0
    res = 1.0
    while it < maxiter:
        q = matvec(p)
        alpha = rz / float(p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        res = float(np.linalg.norm(r)) / bnorm
        if res <= rtol:
            break
        z = r / dv
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    out = np.zeros(n)
    out[idx] = x
    return out, it, res


def exact_parts(row_ptr, col, v, rtol=1e-12):
    """The parts of the large-graph ground truth that one solve each fixes:
    y2[u] = (L_v^{-1} 1)_u / n (zero at v), lvv = (1/n) sum_u y2[u] (= L^+_vv),
    ey2 = (1/2m) d^T L_v^{-1} d (= E[Y2]), and the solver's iterations and
    residuals."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    n = rp.size - 1
    d = (rp[1:] - rp[:-1]).astype(np.float64)
    r1, it1, res1 = solve_lv(row_ptr, col, v, np.ones(n), rtol)
    h, it2, res2 = solve_lv(row_ptr, col, v, d, rtol)
    y2 = r1 / n
    import math
    return {"y2": y2, "lvv": math.fsum(y2.tolist()) / n, "ey2": float(math.fsum((d * h).tolist()) / rp[-1]),
            "hitting": h, "iterations": (it1, it2), "residuals": (res1, res2)}
