"""Learned control variate for the LEWalk estimators (host-side orchestration).

The paper has no control variate.  This module trains the MLP
(8 node features -> 64 -> 64 -> 2) whose outputs become the potentials of the
martingale control variates in include/lap.h (lap_cv_set_potentials), fits
the two coefficients on pilot samples, and applies them.  Every numeric step
runs in the CUDA library: features (lap_features), targets (lap_sample and
lap_hitting_walks), the network's forward/backward on BF16 tensor cores
(lap_mlp_forward, lap_mlp_loss_grad), AdamW (lap_adamw) and the estimators
(lap_cv_estimates).  This module only moves data and chooses hyperparameters.

Targets, produced by the sampler itself on generated graphs:
  head 0: t0(u) = cnt1[u] / omega     (expected Wilson visits, d_u (L_v^{-1})_uu)
  head 1: t1(u) = hit(u) / mean Y2    (hitting time h(u, v) from v-absorbed
                                       walks, divided by E[Y2] = sum pi h)
Potentials:  phi1(w) = pred0(w) / d_w  (~ (L_v^{-1})_ww) for the Wilson draws,
             phi2(w) = pred1(w) * mean Y2 (~ h(w, v)), phi2(v) = 0, for the
             pi-start walks.
"""
from __future__ import annotations

import numpy as np

from .lap import (LAP_MLP_PARAMS, LAP_OPT_CURSOR, LapGraph, lap_adamw, lap_counts, lap_mlp_forward,
                  lap_mlp_loss_grad)

N_FEAT, N_OUT = 8, 2
PILOT_CURSOR = 1 << 31          # pilot sample ids never overlap the estimate's ids


def init_params(seed=0):
    """He-style initialisation of the packed parameter vector (float32, CUDA)."""
    import torch
    rng = np.random.default_rng(seed)
    w1 = rng.standard_normal((64, 8)) * np.sqrt(2.0 / 8)
    w2 = rng.standard_normal((64, 64)) * np.sqrt(2.0 / 64)
    w3 = rng.standard_normal((2, 64)) * np.sqrt(1.0 / 64)
    p = np.concatenate([w1.ravel(), np.zeros(64), w2.ravel(), np.zeros(64), w3.ravel(), np.zeros(2)])
    assert p.size == LAP_MLP_PARAMS
    return torch.tensor(p, dtype=torch.float32, device="cuda")


def training_targets(G: LapGraph, omega=512, reps=16, seed=7):
    """(features [n, 8], targets [n, 2], mask of usable rows) for one graph
    whose root is set; all produced by the library's kernels."""
    import torch
    v = G.root
    G.sample(omega, seed)
    c1, _, sums = lap_counts(G.h, G.n)
    hit = G.hitting_walks(reps, seed + 1).cpu().numpy().astype(np.float64) / reps
    mean_y2 = max(float(sums[2]) / omega, 1e-9)
    t = np.zeros((G.n, 2), dtype=np.float32)
    t[:, 0] = c1.astype(np.float64) / omega
    t[:, 1] = hit / mean_y2
    mask = np.ones(G.n, dtype=bool)
    mask[v] = False
    feats = G.features()
    return feats, torch.from_numpy(t).cuda(), mask


def train(datasets, epochs=8, batch=8192, lr=3e-3, weight_decay=1e-4, seed=0, weights=(1.0, 1.0), log=None):
    """Trains on a list of (features, targets, mask) with AdamW; returns params.
    Minibatches are contiguous slices of a dataset shuffled once on the host."""
    import torch
    X = torch.cat([f[torch.from_numpy(m).cuda()] for f, t, m in datasets]).contiguous()
    T = torch.cat([t[torch.from_numpy(m).cuda()] for f, t, m in datasets]).contiguous()
    perm = torch.from_numpy(np.random.default_rng(seed).permutation(X.shape[0])).cuda()
    X = X[perm].contiguous()
    T = T[perm].contiguous()
    rows = X.shape[0]
    params = init_params(seed)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    grad = torch.zeros_like(params)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    step = 0
    history = []
    for ep in range(epochs):
        lr_ep = lr * 0.5 * (1.0 + np.cos(np.pi * ep / epochs))
        for start in range(0, rows, batch):
            cnt = min(batch, rows - start)
            lap_mlp_loss_grad(params, X[start:], T[start:], cnt, weights[0], weights[1], grad, loss)
            step += 1
            lap_adamw(params, m, v, grad, LAP_MLP_PARAMS, step, lr_ep, weight_decay=weight_decay)
        history.append(float(evaluate(params, X, T, weights)))
        if log:
            log("epoch %d loss %.5f" % (ep, history[-1]))
    return params, history


def evaluate(params, X, T, weights=(1.0, 1.0)):
    import torch
    grad = torch.zeros(LAP_MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    lap_mlp_loss_grad(params, X, T, X.shape[0], weights[0], weights[1], grad, loss)
    return loss.item()


def predict(G: LapGraph, params):
    import torch
    feats = G.features()
    y = torch.empty((G.n, N_OUT), dtype=torch.float32, device="cuda")
    lap_mlp_forward(params, feats, G.n, y)
    return y


def potentials(G: LapGraph, params, mean_y2):
    """phi1 ~ (L_v^{-1})_ww and phi2 ~ h(w, v) from the network (float64, CUDA)."""
    import torch
    y = predict(G, params).double()
    deg = torch.from_numpy(np.diff(G.row_ptr_host.astype(np.int64)).astype(np.float64)).cuda()
    phi1 = (y[:, 0] / deg).contiguous()
    phi2 = (y[:, 1] * float(mean_y2)).contiguous()
    phi2[G.root] = 0.0
    return phi1, phi2


def pilot_mean_y2(G: LapGraph, seed, samples=2048):
    """Mean pi-start walk length E[Y2] from pilot samples whose ids (from
    PILOT_CURSOR + 2^30) are disjoint from both the estimate's and fit_betas';
    resets the root (counts and cursor) afterwards."""
    root = G.root
    G.set_root(root)
    G.set_option(LAP_OPT_CURSOR, PILOT_CURSOR + (1 << 30))
    _, y2 = G.sample_trace(samples, seed)
    G.set_root(root)
    return float(y2.double().mean().item())


def fit_betas(G: LapGraph, phi1, phi2, seed, pilot=4096, batches=8):
    """Coefficients from pilot samples (ids from PILOT_CURSOR, disjoint from the
    estimate's): beta2 minimises Var(Y1 - Y2 + beta2 M2) over per-sample
    traces; beta1 pools, over nodes, per-node covariances of the visit count
    with Z1/d between `batches` independent pilot batches."""
    import torch
    root = G.root
    G.set_root(root)
    G.set_option(LAP_OPT_CURSOR, PILOT_CURSOR)
    G.cv_set_potentials(phi1, phi2)
    d = np.diff(G.row_ptr_host.astype(np.int64)).astype(np.float64)
    per = max(1, pilot // batches)
    ys, ms = [], []
    prev_c1 = np.zeros(G.n)
    prev_a1 = np.zeros(G.n)
    vis, zed = [], []
    from .lap import lap_counts as counts
    s1 = None
    for b in range(batches):
        y1, y2, m2 = G.sample_trace_cv(per, seed)
        ys.append((y1 - y2).double().cpu().numpy())
        ms.append(m2.cpu().numpy())
        c1, _, _ = counts(G.h, G.n)
        a1, _, _ = G.cv_sums()
        c1 = c1.astype(np.float64)
        a1 = a1.astype(np.float64)
        if s1 is None:
            s1 = _neighbour_sum_host(G, phi1)
        dc1 = c1 - prev_c1
        da1 = a1 - prev_a1
        prev_c1, prev_a1 = c1, a1
        vis.append(dc1)
        zed.append((d * da1 - dc1 * s1) / d)
    y = np.concatenate(ys)
    m = np.concatenate(ms)
    c = np.cov(y, m)
    beta2 = -c[0, 1] / c[1, 1] if c[1, 1] > 0 else 0.0
    V = np.array(vis)
    Z = np.array(zed)
    Vc = V - V.mean(axis=0)
    Zc = Z - Z.mean(axis=0)
    num = float(np.sum(Vc * Zc))
    den = float(np.sum(Zc * Zc))
    beta1 = num / den if den > 0 else 0.0
    G.set_root(root)
    return float(beta1), float(beta2)


def _neighbour_sum_host(G, phi1):
    h = np.rint(np.ldexp(phi1.cpu().numpy(), 16)).astype(np.int64)
    rp = G.row_ptr_host.astype(np.int64)
    src = np.repeat(np.arange(G.n), rp[1:] - rp[:-1])
    out = np.zeros(G.n, dtype=np.int64)
    np.add.at(out, src, h[G.col_host])
    return out.astype(np.float64)
