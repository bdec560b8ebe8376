"""Oracle for the learned control variate (CV) of the LEWalk estimators.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py): plain numpy, FP64.

The paper has no control variate; this is the CPU statement of what the GPU
library computes for it:

* node features (8 per node, local to the node and the root v),
* the MLP 8 -> 64 -> 64 -> 2 (ReLU), its MSE loss, gradients and AdamW step,
  with the GPU kernels' BF16 rounding points emulated (inputs, weights and
  hidden activations rounded to BF16, everything else FP64),
* integer potentials and the martingale control-variate estimators.

Martingale terms.  For an integer potential h on nodes and S[u] = sum of h
over N(u), every random step u -> w (w uniform on N(u)) contributes
xi = d_u h[w] - S[u], whose mean given u is exactly zero.  Summing xi over
Wilson draws at u gives Z1[u] = d_u A1[u] - cnt1[u] S1[u] (A1[u] = sum of
h1[w] over the draws at u); summing xi / d_u over the steps of the pi-start
walks gives M2 = sum_u (d_u A2[u] - P2[u] S2[u]) / d_u.  The estimators
    y1_cv(u) = (cnt1[u] - beta1 Z1[u] / d_u) / (omega d_u)          (ECC, Alg. 2)
    kappa_cv = (sum Y1 - sum Y2 + beta2 M2) / omega                  (KC, Alg. 4)
stay unbiased for any potential and any beta chosen independently of the
samples.  With h2 equal to the hitting time h(., v), Y2 - M2 reduces to the
hitting time of the start node (the walk length's randomness cancels).
"""
from __future__ import annotations

import numpy as np

N_FEAT = 8
HIDDEN = 64
N_OUT = 2
FIXED_POINT_BITS = 16


# ------------------------------------------------------------------- features

def bfs_hops(row_ptr, col, v):
    n = len(row_ptr) - 1
    hops = np.full(n, -1, dtype=np.int64)
    hops[v] = 0
    frontier = [v]
    while frontier:
        nxt = []
        for u in frontier:
            for w in col[row_ptr[u]:row_ptr[u + 1]]:
                if hops[w] < 0:
                    hops[w] = hops[u] + 1
                    nxt.append(int(w))
        frontier = nxt
    return hops


def features(row_ptr, col, v, absorb_iters=8):
    """8 features per node (float64):
      f0 ln d_u                      f4 ln(mean degree of the neighbours)
      f1 1 / d_u                     f5 share of neighbours of degree 1
      f2 ln(1 + hop distance to v)   f6 ln(two-hop degree sum / one-hop degree sum)
      f3 1 if u is a neighbour of v  f7 P(walk from u hits v within 8 steps)
    """
    rp = np.asarray(row_ptr, dtype=np.int64)
    cl = np.asarray(col, dtype=np.int64)
    n = rp.size - 1
    d = (rp[1:] - rp[:-1]).astype(np.float64)
    src = np.repeat(np.arange(n), rp[1:] - rp[:-1])
    s1 = np.bincount(src, weights=d[cl], minlength=n)              # sum of neighbour degrees
    s2 = np.bincount(src, weights=s1[cl], minlength=n)             # two-hop degree sum
    ones = np.bincount(src, weights=(d[cl] == 1.0).astype(np.float64), minlength=n)
    hops = bfs_hops(rp, cl, v)
    adj_v = np.zeros(n)
    adj_v[cl[rp[v]:rp[v + 1]]] = 1.0
    a = np.zeros(n)
    a[v] = 1.0
    for _ in range(absorb_iters):
        a = np.bincount(src, weights=a[cl], minlength=n) / d
        a[v] = 1.0
    f = np.empty((n, N_FEAT))
    f[:, 0] = np.log(d)
    f[:, 1] = 1.0 / d
    f[:, 2] = np.log1p(hops)
    f[:, 3] = adj_v
    f[:, 4] = np.log(s1 / d)
    f[:, 5] = ones / d
    f[:, 6] = np.log(s2 / s1)
    f[:, 7] = a
    return f


# ------------------------------------------------------------------------ MLP

def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    rounded = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(x))


def init_params(seed=0):
    """He-style initialisation: W1 [64, 8], W2 [64, 64], W3 [2, 64], biases zero."""
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.standard_normal((HIDDEN, N_FEAT)) * np.sqrt(2.0 / N_FEAT),
        "b1": np.zeros(HIDDEN),
        "W2": rng.standard_normal((HIDDEN, HIDDEN)) * np.sqrt(2.0 / HIDDEN),
        "b2": np.zeros(HIDDEN),
        "W3": rng.standard_normal((N_OUT, HIDDEN)) * np.sqrt(1.0 / HIDDEN),
        "b3": np.zeros(N_OUT),
    }


def forward(params, x, quantize=True):
    """Returns (y [N, 2], cache).  quantize=True rounds x, the weights and both
    hidden activations to BF16 where the GPU feeds them to the tensor cores."""
    q = bf16 if quantize else (lambda t: np.asarray(t, dtype=np.float64))
    xb, W1, W2, W3 = q(x), q(params["W1"]), q(params["W2"]), q(params["W3"])
    z1 = xb @ W1.T + params["b1"]
    h1 = q(np.maximum(z1, 0.0))
    z2 = h1 @ W2.T + params["b2"]
    h2 = q(np.maximum(z2, 0.0))
    y = h2 @ W3.T + params["b3"]
    return y, (xb, W1, W2, W3, z1, h1, z2, h2)


def loss_and_grads(params, x, t, w=(1.0, 1.0), quantize=True):
    """MSE loss (1/N) sum_i sum_k w_k (y_ik - t_ik)^2 and its gradients.

    quantize=True states the BF16 training arithmetic: every operand of a
    product (a tensor-core operand on the GPU) is BF16, sums are exact here
    (FP32 there).  Besides the forward pass's rounding points, the backward
    pass rounds the output error dY and the back-propagated errors dH2, dH1
    to BF16 where they enter a product (the weight gradients dY^T H2,
    dH2^T H1, dH1^T X and the propagations dY W3, dH2 W2); the bias
    gradients sum the unrounded errors."""
    y, (xb, W1, W2, W3, z1, h1, z2, h2) = forward(params, x, quantize)
    q = bf16 if quantize else (lambda a: a)
    wk = np.asarray(w, dtype=np.float64)
    nrow = x.shape[0]
    r = y - t
    loss = float(np.sum(wk * r * r) / nrow)
    dy = 2.0 * wk * r / nrow
    dyq = q(dy)
    g = {"W3": dyq.T @ h2, "b3": dy.sum(axis=0)}
    dh2 = (dyq @ W3) * (z2 > 0)
    dh2q = q(dh2)
    g["W2"] = dh2q.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2q @ W2) * (z1 > 0)
    g["W1"] = q(dh1).T @ xb
    g["b1"] = dh1.sum(axis=0)
    return loss, g


def adamw_step(w, m, v, g, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """AdamW (Loshchilov & Hutter, decoupled weight decay).  Returns new (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    w = w - lr * (mh / (np.sqrt(vh) + eps) + wd * w)
    return w, m, v


# ----------------------------------------------------------- CV estimators

def quantize_potential(phi, bits=FIXED_POINT_BITS):
    """Integer potential h = round(2^bits * phi) (int64)."""
    return np.rint(np.ldexp(np.asarray(phi, dtype=np.float64), bits)).astype(np.int64)


def neighbour_sums(row_ptr, col, h):
    rp = np.asarray(row_ptr, dtype=np.int64)
    n = rp.size - 1
    src = np.repeat(np.arange(n), rp[1:] - rp[:-1])
    return _exact_sum(src, np.asarray(h, dtype=np.int64)[np.asarray(col)], n)


def _exact_sum(idx, vals, n):
    out = np.zeros(n, dtype=np.int64)
    np.add.at(out, idx, vals.astype(np.int64))
    return out


def martingale_z1(row_ptr, col, h1, cnt1, a1):
    """Z1[u] = d_u A1[u] - cnt1[u] S1[u] (exact int64)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    d = rp[1:] - rp[:-1]
    s1 = neighbour_sums(row_ptr, col, h1)
    return d * np.asarray(a1, dtype=np.int64) - np.asarray(cnt1, dtype=np.int64) * s1


def martingale_m2(row_ptr, col, h2, a2, p2):
    """M2 = sum_u (d_u A2[u] - P2[u] S2[u]) / d_u (compensated FP64 sum)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    d = rp[1:] - rp[:-1]
    s2 = neighbour_sums(row_ptr, col, h2)
    terms = (d * np.asarray(a2, dtype=np.int64) - np.asarray(p2, dtype=np.int64) * s2).astype(np.float64) / d
    import math
    return math.fsum(terms.tolist())


def finalize_cv(row_ptr, v, omega, cnt1, cnt2, sum_y1, sum_y2, z1, m2, beta1, beta2):
    """Returns (ldiag, ecc, kemeny) of the CV estimators (FP64)."""
    import math
    rp = np.asarray(row_ptr, dtype=np.int64)
    n = rp.size - 1
    d = (rp[1:] - rp[:-1]).astype(np.float64)
    w = float(omega)
    c1 = np.asarray(cnt1, dtype=np.float64) - beta1 * (np.asarray(z1, dtype=np.float64) / d)
    y1 = c1 / (w * d)
    y2 = np.asarray(cnt2, dtype=np.float64) / (w * d)
    lvv = math.fsum(y2.tolist()) / n
    ld = (y1 - 2.0 * y2) + lvv
    ld[v] = lvv
    tr = math.fsum(ld.tolist())
    ecc = (n - 1) / (n * ld + tr)
    kc = ((float(sum_y1) - float(sum_y2)) + beta2 * m2) / w
    return ld, ecc, kc


# ------------------------------------------- training targets and coefficients

def training_targets(cnt1, omega, hit_sums, reps, sum_y2, v):
    """Targets of the network's two heads for one graph (float32 [n, 2]):
    t0(u) = cnt1(u) / omega, the mean number of Wilson visits of u, whose
    expectation is d_u (L_v^{-1})_uu (Section 3.4, LE-walk lemma); t1(u) =
    (hit_sums(u) / reps) / Ybar2 with Ybar2 = max(sum_y2 / omega, 1e-9), the
    mean v-absorbed walk length from u (expectation h(u, v), Section 3.2)
    over the estimate of E[Y2] = sum_u pi(u) h(u, v).  FP64, then rounded to
    float32; the root's row is zero."""
    c1 = np.asarray(cnt1, dtype=np.float64)
    hit = np.asarray(hit_sums, dtype=np.float64)
    mean_y2 = float(sum_y2) / float(omega)
    if not mean_y2 > 1e-9:
        mean_y2 = 1e-9
    t = np.zeros((c1.size, 2), dtype=np.float64)
    t[:, 0] = c1 / float(omega)
    t[:, 1] = (hit / float(reps)) / mean_y2
    t[v] = 0.0
    return t.astype(np.float32)


def potentials(y, row_ptr, v, scale2):
    """Potentials from the network's outputs y [n, 2] (float32): phi1(u) =
    y0(u) / d_u (the predicted visits per unit degree, ~ (L_v^{-1})_uu) and
    phi2(u) = y1(u) * scale2 (the predicted hitting time; scale2 is the mean
    pi-walk length the targets were divided by), phi2(v) = 0."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    d = (rp[1:] - rp[:-1]).astype(np.float64)
    yy = np.asarray(y, dtype=np.float32).astype(np.float64)
    phi1 = yy[:, 0] / d
    phi2 = yy[:, 1] * float(scale2)
    phi2[v] = 0.0
    return phi1, phi2


def betas_from_batches(V, Z, y, m):
    """Least-squares coefficients of the two control variates.

    V, Z: [batches, n] per-batch visits V_bu and martingale sums Z_bu =
    Z1_b(u) / d_u.  The ECC estimator uses cnt1 - beta1 Z1/d, so beta1 is the
    regression slope of V on Z pooled over nodes, each node centred on its
    own batch mean: beta1 = sum_u cov_b(V_u, Z_u) / sum_u var_b(Z_u).
    y, m: per-sample Y1 - Y2 and M2.  The Kemeny estimator uses y + beta2 m,
    so beta2 = -cov(y, m) / var(m).  A zero denominator gives 0."""
    V = np.asarray(V, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    Vc = V - V.mean(axis=0)
    Zc = Z - Z.mean(axis=0)
    den1 = float(np.sum(Zc * Zc))
    beta1 = float(np.sum(Vc * Zc)) / den1 if den1 > 0 else 0.0
    c = np.cov(np.asarray(y, dtype=np.float64), np.asarray(m, dtype=np.float64))
    beta2 = -float(c[0, 1]) / float(c[1, 1]) if c[1, 1] > 0 else 0.0
    return beta1, beta2


def fit_betas(row_ptr, col, v, seed, first, per, batches, h1, h2):
    """The coefficients from `batches` pilot batches of `per` samples with ids
    first + b * per + [0, per) (the CPU sampler with both potentials), by
    betas_from_batches."""
    import oracle
    rp = np.asarray(row_ptr, dtype=np.int64)
    d = rp[1:] - rp[:-1]
    V, Z, ys, ms = [], [], [], []
    for b in range(batches):
        cnt, a1, _, _, m2 = oracle.sample_cv(row_ptr, col, v, seed, first + b * per, per, h1=h1, h2=h2)
        z1 = martingale_z1(row_ptr, col, h1, cnt.cnt1, a1)
        V.append(cnt.cnt1.astype(np.float64))
        Z.append(z1.astype(np.float64) / d)
        ys.append(cnt.y1.astype(np.int64) - cnt.y2.astype(np.int64))
        ms.append(m2)
    V, Z = np.array(V), np.array(Z)
    V[:, v] = 0.0
    Z[:, v] = 0.0
    return betas_from_batches(V, Z, np.concatenate(ys), np.concatenate(ms))
