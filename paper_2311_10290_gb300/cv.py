"""Learned control variate for the LEWalk estimators (host-side orchestration).

The paper has no control variate.  This module trains the MLP
(8 node features -> 64 -> 64 -> 2) whose outputs become the potentials of the
martingale control variates in include/lap.h (lap_cv_set_potentials), fits
the two coefficients on pilot samples, and applies them.  It only sequences
calls of the CUDA library and moves data between them; every value of the
method is computed there: features (lap_features), training targets
(lap_sample, lap_cv_targets), the network's forward/backward on BF16 tensor
cores (lap_mlp_forward, lap_mlp_loss_grad), AdamW (lap_adamw), potentials
(lap_cv_potentials), coefficients (lap_cv_fit_betas) and the estimators
(lap_cv_estimates).  What stays here: the training schedule (epochs,
minibatches of a once-shuffled row order, a cosine learning rate) and the
parameter initialisation.

Targets, produced by the sampler itself on generated graphs (lap_cv_targets):
  head 0: cnt1[u] / omega     (expected Wilson visits, d_u (L_v^{-1})_uu)
  head 1: hit(u) / mean Y2    (hitting time h(u, v) from v-absorbed walks,
                               divided by the estimate of E[Y2] = sum pi h)
Potentials (lap_cv_potentials): phi1 = pred0 / d (~ (L_v^{-1})_ww) for the
Wilson draws, phi2 = pred1 * mean Y2 (~ h(w, v)), phi2(v) = 0, for the
pi-start walks.
"""
from __future__ import annotations

import numpy as np

from .lap import LAP_MLP_PARAMS, LAP_OPT_CURSOR, LapGraph, lap_adamw, lap_mlp_forward, lap_mlp_loss_grad

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
    whose root is set; all produced by the library's kernels.  The root's
    row is left out (its targets are zero by definition)."""
    G.sample(omega, seed)
    t = G.cv_targets(reps, seed + 1)
    mask = np.ones(G.n, dtype=bool)
    mask[G.root] = False
    return G.features(), t, mask


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


def pilot_potentials(G: LapGraph, params, seed, samples=2048):
    """phi1 ~ (L_v^{-1})_ww and phi2 ~ h(w, v) (float64 CUDA tensors) from the
    network, phi2 scaled by the mean pi-walk length of `samples` pilot samples
    whose ids (from PILOT_CURSOR + 2^30) are disjoint from both the estimate's
    and fit_betas'; resets the root (counts and cursor) afterwards."""
    root = G.root
    G.set_root(root)
    G.set_option(LAP_OPT_CURSOR, PILOT_CURSOR + (1 << 30))
    G.sample(samples, seed)
    phi1, phi2 = G.cv_potentials(predict(G, params))
    G.set_root(root)
    return phi1, phi2


def fit_betas(G: LapGraph, phi1, phi2, seed, pilot=4096, batches=8):
    """Coefficients from pilot samples (ids from PILOT_CURSOR, disjoint from the
    estimate's), computed by lap_cv_fit_betas: beta2 minimises the variance of
    Y1 - Y2 + beta2 M2 over the per-sample traces; beta1 pools, over nodes,
    per-node covariances of the visit count with Z1/d between `batches`
    pilot batches.  Leaves the handle reset with the potentials set."""
    return G.cv_fit_betas(phi1, phi2, seed, PILOT_CURSOR, pilot, batches)
