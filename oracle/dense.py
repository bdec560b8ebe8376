"""Dense FP64 estimand for the LEWalk estimators (arXiv 2311.10290).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg, never by the library.

Everything here is the plain definition written out with numpy linear algebra
on dense matrices, so it is only meant for graphs of up to a few thousand nodes.

* ``L = D - A`` and ``P = D^{-1} A``, ``pi(u) = d_u / 2m``          (Section 2)
* ``L^+`` the Moore-Penrose pseudo-inverse                          (Section 2)
* electrical closeness ``c(u) = (n-1) / (n L^+_uu + Tr L^+)``       (Section 2, ECC)
* Kemeny's constant ``kappa = Tr(calL^+) = sum_{i>=2} 1/sigma_i``   (Section 2, KC)
* ``L_v`` = ``L`` without row and column ``v``; its inverse gives the quantities the
  samplers estimate (Section 3.2, Lemma "v-absorbed walk"; Section 3.4, Lemma
  "Loop-erased walk"; Alg. 2 and Alg. 4):

  - ``E[visits of u in one LE_v run] = (I - P_v)^{-1}_uu = d_u (L_v^{-1})_uu``
  - ``E[passes of u in a walk from uniform s] = d_u (1/n) e_u^T L_v^{-1} 1``
  - ``E[Y1] = Tr((I - P_v)^{-1})``,   ``E[Y2] = (1/2m) d_v^T L_v^{-1} d_v``
"""
from __future__ import annotations

import numpy as np


def adjacency(n, row_ptr, col):
    """Dense 0/1 adjacency matrix of a CSR graph."""
    a = np.zeros((n, n), dtype=np.float64)
    rp = np.asarray(row_ptr, dtype=np.int64)
    c = np.asarray(col, dtype=np.int64)
    for u in range(n):
        a[u, c[rp[u]:rp[u + 1]]] = 1.0
    return a


def laplacian(n, row_ptr, col):
    """Combinatorial Laplacian L = D - A (Section 2)."""
    a = adjacency(n, row_ptr, col)
    return np.diag(a.sum(axis=1)) - a


def degrees(n, row_ptr):
    rp = np.asarray(row_ptr, dtype=np.int64)
    return (rp[1:] - rp[:-1]).astype(np.float64)


def pinv_laplacian(n, row_ptr, col):
    """L^+ = sum_{i>=2} u_i u_i^T / lambda_i from the eigendecomposition (Section 2)."""
    lam, vec = np.linalg.eigh(laplacian(n, row_ptr, col))
    inv = np.zeros_like(lam)
    inv[1:] = 1.0 / lam[1:]          # lambda_1 = 0 for a connected graph
    return (vec * inv) @ vec.T


def ecc(n, row_ptr, col):
    """Electrical closeness c(u) = (n-1) / (n L^+_uu + Tr L^+) (Section 2)."""
    lp = pinv_laplacian(n, row_ptr, col)
    dg = np.diag(lp)
    return (n - 1) / (n * dg + dg.sum())


def kirchhoff(n, row_ptr, col):
    """Kirchhoff index as Section 5 ("Discussions") defines it: Tr(L^+)."""
    return float(np.trace(pinv_laplacian(n, row_ptr, col)))


def rw_betweenness(n, row_ptr, col):
    """Random-walk betweenness as Section 5 ("Discussions") states it:
    c_b(u) = 1/n + Tr(L^+) / ((n-1) (Tr(L^+) + n L^+_uu))."""
    dg = np.diag(pinv_laplacian(n, row_ptr, col))
    return from_ldiag(dg)[1]


def from_ldiag(ldiag):
    """(Kirchhoff index, random-walk betweenness) from a vector of L^+_uu
    (Section 5, "Discussions"); the trace is a compensated FP64 sum."""
    import math
    ld = np.asarray(ldiag, dtype=np.float64)
    n = ld.size
    tr = math.fsum(ld.tolist())
    return tr, 1.0 / n + tr / ((n - 1) * (tr + n * ld))


def kemeny(n, row_ptr, col):
    """kappa(G) = Tr(calL^+) = sum over the nonzero eigenvalues sigma of
    calL = I - D^{-1/2} A D^{-1/2} of 1/sigma (Section 2, KC)."""
    a = adjacency(n, row_ptr, col)
    dm = 1.0 / np.sqrt(a.sum(axis=1))
    nl = np.eye(n) - (dm[:, None] * a) * dm[None, :]
    sig = np.linalg.eigvalsh(nl)
    return float(np.sum(1.0 / sig[1:]))


def lv_inverse(n, row_ptr, col, v):
    """(L_v)^{-1} as an n x n matrix with zeros in row and column v."""
    lap = laplacian(n, row_ptr, col)
    keep = np.array([u for u in range(n) if u != v], dtype=np.int64)
    inv = np.linalg.inv(lap[np.ix_(keep, keep)])
    out = np.zeros((n, n))
    out[np.ix_(keep, keep)] = inv
    return out


def expectations(n, row_ptr, col, v):
    """Per-sample expectations of what one sample id adds (Alg. 2, Alg. 4).

    Returns a dict with
      visits[u]  E[visits of u in one Wilson run]             = d_u (L_v^{-1})_uu
      passes[u]  E[passes of u in the uniform-start walk]     = d_u (1/n) (L_v^{-1} 1)_u
      y1         E[Y1] = Tr((I-P_v)^{-1})
      y2         E[Y2] = (1/2m) d^T L_v^{-1} d
      lvinv      L_v^{-1} (zero row/col v)
    """
    d = degrees(n, row_ptr)
    li = lv_inverse(n, row_ptr, col, v)
    visits = d * np.diag(li)
    passes = d * (li.sum(axis=1) / n)
    two_m = d.sum()
    return {
        "visits": visits,
        "passes": passes,
        "y1": float(visits.sum()),
        "y2": float(d @ li @ d / two_m),
        "lvinv": li,
    }


def ldag_from_lv(n, lvinv, v):
    """L^+ from L_v^{-1} by the element-wise identities (Section 3.1, Thm 1 and
    the four cases that follow it): with r = L_v^{-1} 1 and S = 1^T L_v^{-1} 1,
      L^+_st = (L_v^{-1})_st - r_s/n - r_t/n + S/n^2   (s, t != v)
      L^+_sv = -r_s/n + S/n^2                          (s != v)
      L^+_vv = S/n^2
    lvinv is n x n with zero row and column v, so one formula covers all cases."""
    r = lvinv.sum(axis=1)
    s = r.sum()
    return lvinv - r[:, None] / n - r[None, :] / n + s / n ** 2


def hitting_times_to(n, row_ptr, col, v):
    """h(u, v) for all u: h = (I - P_v)^{-1} 1 = L_v^{-1} d (Lemma "v-absorbed walk")."""
    d = degrees(n, row_ptr)
    return lv_inverse(n, row_ptr, col, v) @ d
