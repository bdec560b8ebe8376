"""GPU parity of the learned control variate with its oracle (oracle/cv.py,
oracle_sample_cv, oracle_hitting_walks), and its measured gain.

Integer sums (A1, A2, P2, hitting-walk lengths) and per-sample M2 are
bit-exact; CV estimates agree to 1e-12 relative; features to 1e-5; the BF16
MLP forward outputs and gradient entries agree element by element with the
oracle (same BF16 rounding points, see assert_elementwise) for both MLP
kernels (tcgen05 with TMEM accumulators, and mma.sync), the loss to 1e-3;
AdamW (FP32) to 1e-5."""
import numpy as np
import pytest

import oracle
import oracle.cv as CV
import oracle.dense as D
from paper_2311_10290_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from paper_2311_10290_gb300 import cv as CVG  # noqa: E402
from paper_2311_10290_gb300.lap import (LAP_MLP_MMA_SYNC, LAP_MLP_PARAMS, LAP_MLP_TCGEN05, LAP_OPT_KERNEL,  # noqa: E402
                                        LAP_OPT_PATHS, LAP_OPT_STACK, LAP_OPT_WALKERS, LAP_STAT_FALLBACKS,
                                        LAP_STAT_LAST_KERNEL, LapGraph, lap_adamw, lap_mlp_forward,
                                        lap_mlp_loss_grad, lap_mlp_select)


def packed(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["W3"].ravel(), p["b3"]])


def unpack(v):
    v = np.asarray(v, dtype=np.float64)
    o = 0
    out = {}
    for k, shp in [("W1", (64, 8)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("W3", (2, 64)), ("b3", (2,))]:
        sz = int(np.prod(shp))
        out[k] = v[o:o + sz].reshape(shp)
        o += sz
    return out


@pytest.mark.parametrize("g", [I.ba(5000, 3, seed=1), I.rmat(10, 6, seed=2), I.er(800, 0.01, seed=3)],
                         ids=["ba", "rmat", "er"])
def test_features_match_oracle(g):
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 26)
    try:
        v = G.set_root()
        f = G.features().cpu().numpy().astype(np.float64)
    finally:
        G.close()
    ref = CV.features(g.row_ptr, g.col, v)
    np.testing.assert_allclose(f, ref.astype(np.float32).astype(np.float64), rtol=2e-6, atol=1e-6)


def test_hitting_walks_bit_exact():
    g = I.ba(2000, 3, seed=4)
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 26)
    try:
        v = G.set_root()
        s = G.hitting_walks(7, 99).cpu().numpy().astype(np.uint64)
    finally:
        G.close()
    assert np.array_equal(s, oracle.hitting_walks(g.row_ptr, g.col, v, 99, 7))


def _cv_run(g, root, seed, omega, phi1, phi2, kernel=None, splits=None, paths=False, walkers=0, stack=0):
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 28)
    try:
        if kernel:
            G.set_option(LAP_OPT_KERNEL, kernel)
        if paths:
            G.set_option(LAP_OPT_PATHS, 1)
        if walkers:
            G.set_option(LAP_OPT_WALKERS, walkers)
        if stack:
            G.set_option(LAP_OPT_STACK, stack)
        v = G.set_root(root)
        G.cv_set_potentials(None if phi1 is None else torch.from_numpy(phi1).cuda(),
                            None if phi2 is None else torch.from_numpy(phi2).cuda())
        for part in splits or [omega]:
            G.sample(part, seed)
        c1, c2, s = G.counts()
        a1, a2, p2 = G.cv_sums()
        ld, ec, kc, m2 = G.cv_estimates(0.9, 1.1)
        return dict(v=v, c1=c1, c2=c2, s=s, a1=a1, a2=a2, p2=p2, ld=ld, ec=ec, kc=kc, m2=m2,
                    kernel=G.stat(LAP_STAT_LAST_KERNEL), fallbacks=G.stat(LAP_STAT_FALLBACKS))
    finally:
        G.close()


@pytest.mark.parametrize("paths", [False, True], ids=["own_draws", "stack_paths"])
@pytest.mark.parametrize("kernel", [1, 2, 3], ids=["wide", "compact", "group"])
@pytest.mark.parametrize("name,maker,root", [("ba", lambda: I.ba(3000, 3, seed=5), -1),
                                             ("rmat", lambda: I.rmat(9, 8, seed=6), -1),
                                             ("path_counts_table", lambda: I.path(50), 0),
                                             ("path_table_heavy", lambda: I.path(256), 255)],
                         ids=["ba", "rmat", "path_counts_table", "path_table_heavy"])
def test_cv_sums_and_estimates_match_oracle(name, maker, root, kernel, paths):
    g = maker()
    rng = np.random.default_rng(3)
    phi1 = rng.uniform(0.0, 3.0, g.n)
    phi2 = rng.uniform(0.0, 50.0, g.n)
    r = _cv_run(g, root, 17, 300, phi1, phi2, kernel=kernel, splits=[100, 200], paths=paths)
    assert r["kernel"] == kernel
    _check_cv(g, r, phi1, phi2, 17, 300, paths)


@pytest.mark.parametrize("paths", [False, True], ids=["own_draws", "stack_paths"])
@pytest.mark.parametrize("walkers", [2, 4, 8, 16])
def test_cv_group_kernel_withdrawn_samples_are_rerun_exactly(walkers, paths):
    """Kernel 3 with a 16-entry stack per walker on a path graph rooted at
    one end: samples are withdrawn (their repeat visits and the potentials of
    all their Wilson draws subtracted, and with loop-included paths their
    departures and pi-path terms) and re-run with kernel 1; every CV sum
    stays bit-exact."""
    g = I.path(200)
    rng = np.random.default_rng(8)
    phi1 = rng.uniform(0.0, 3.0, g.n)
    phi2 = rng.uniform(0.0, 50.0, g.n)
    r = _cv_run(g, 0, 23, 64, phi1, phi2, kernel=3, walkers=walkers, stack=16, paths=paths)
    assert r["fallbacks"] > 0
    _check_cv(g, r, phi1, phi2, 23, 64, paths)


@pytest.mark.parametrize("walkers", [4, 16])
def test_cv_group_kernel_paths_departure_cap(walkers):
    """Kernel 3, loop-included paths and the control variate on a path graph
    rooted at one end (the samples of test_group_kernel_paths_departure_cap_*:
    some paths leave a node 255 times): withdrawn samples give back their
    path departures and the pi path's A2 and P2 terms; every sum bit-exact."""
    g = I.path(200)
    rng = np.random.default_rng(10)
    phi1 = rng.uniform(0.0, 3.0, g.n)
    phi2 = rng.uniform(0.0, 50.0, g.n)
    r = _cv_run(g, 0, 19, 48, phi1, phi2, kernel=3, walkers=walkers, paths=True)
    assert r["kernel"] == 3 and r["fallbacks"] > 0
    _check_cv(g, r, phi1, phi2, 19, 48, True)


@pytest.mark.parametrize("walkers", [8, 16])
def test_cv_group_kernel_rmat(walkers):
    g = I.rmat(12, 8, seed=3)
    rng = np.random.default_rng(9)
    phi1 = rng.uniform(0.0, 3.0, g.n)
    phi2 = rng.uniform(0.0, 50.0, g.n)
    r = _cv_run(g, -1, 31, 500, phi1, phi2, kernel=3, walkers=walkers, splits=[123, 377])
    assert r["kernel"] == 3
    _check_cv(g, r, phi1, phi2, 31, 500, False)


def _check_cv(g, r, phi1, phi2, seed, omega, paths):
    v = r["v"]
    h1, h2 = CV.quantize_potential(phi1), CV.quantize_potential(phi2)
    cnt, a1, a2, p2, m2 = oracle.sample_cv(g.row_ptr, g.col, v, seed, 0, omega, h1=h1, h2=h2, paths=paths)
    assert np.array_equal(r["c1"], cnt.cnt1) and np.array_equal(r["c2"], cnt.cnt2)
    assert np.array_equal(r["a1"], a1) and np.array_equal(r["a2"], a2) and np.array_equal(r["p2"], p2)
    z1 = CV.martingale_z1(g.row_ptr, g.col, h1, cnt.cnt1, a1)
    m2t = CV.martingale_m2(g.row_ptr, g.col, h2, a2, p2)
    assert r["m2"] == pytest.approx(m2t, rel=1e-12, abs=1e-6)
    ld, ec, kc = CV.finalize_cv(g.row_ptr, v, omega, cnt.cnt1, cnt.cnt2, cnt.sum_y1, cnt.sum_y2, z1, m2t, 0.9, 1.1)
    np.testing.assert_allclose(r["ld"], ld, rtol=1e-12)
    np.testing.assert_allclose(r["ec"], ec, rtol=1e-12)
    assert r["kc"] == pytest.approx(kc, rel=1e-12)


@pytest.mark.parametrize("kernel", [2, 3])
def test_per_sample_m2_trace_bit_exact(kernel):
    g = I.ba(4000, 4, seed=8)
    phi2 = np.random.default_rng(5).uniform(0.0, 30.0, g.n)
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 27)
    try:
        G.set_option(LAP_OPT_KERNEL, kernel)
        v = G.set_root()
        G.cv_set_potentials(None, torch.from_numpy(phi2).cuda())
        y1, y2, m2 = G.sample_trace_cv(64, 3)
        torch.cuda.synchronize()
        assert G.stat(LAP_STAT_LAST_KERNEL) == kernel
    finally:
        G.close()
    cnt, a1, a2, p2, m2o = oracle.sample_cv(g.row_ptr, g.col, v, 3, 0, 64, h2=CV.quantize_potential(phi2))
    assert np.array_equal(y1.cpu().numpy().astype(np.uint64), cnt.y1)
    assert np.array_equal(y2.cpu().numpy().astype(np.uint64), cnt.y2)
    assert np.array_equal(m2.cpu().numpy(), m2o)


def assert_elementwise(got, ref, axis, what=""):
    """Element-wise bound of the BF16 MLP against the FP64 oracle with the
    same BF16 rounding points: |got - ref| <= 1e-2 |ref| + 2e-3 rms, the rms
    taken per output column (axis=0) or per parameter tensor (axis=None).
    Both sides round the inputs, weights and hidden activations to BF16 at
    the same points, so they differ only by FP32 accumulation order (about
    1e-7 relative per sum) and the rare hidden value whose FP32 and FP64
    pre-activations round to neighbouring BF16 values (one BF16 ulp, 2^-8
    relative, weighted by an outgoing weight of about 0.1-0.2: about 5e-4 of
    the column's rms per such value).  A wrong tile, fragment or column
    gives errors of the order of the rms itself."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    rms = np.sqrt(np.mean(ref * ref, axis=axis, keepdims=axis is not None))
    bad = np.abs(got - ref) > 1e-2 * np.abs(ref) + 2e-3 * rms
    assert not np.any(bad), (what, np.argwhere(bad)[:5], np.max(np.abs(got - ref) / (np.abs(ref) + rms)))


def _params(seed):
    p = CV.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    p["b1"] = 0.1 * rng.standard_normal(64)
    p["b2"] = 0.1 * rng.standard_normal(64)
    p["b3"] = 0.1 * rng.standard_normal(2)
    return p


@pytest.fixture(params=[LAP_MLP_TCGEN05, LAP_MLP_MMA_SYNC], ids=["tcgen05", "mma_sync"])
def mlp_kernel(request):
    lap_mlp_select(request.param)
    yield request.param
    lap_mlp_select(LAP_MLP_TCGEN05)


@pytest.mark.parametrize("rows", [1, 17, 64, 127, 128, 129, 1000, 4099, 100_003])
def test_mlp_forward_matches_oracle(rows, mlp_kernel):
    p = _params(1)
    x = np.random.default_rng(2).standard_normal((rows, 8)).astype(np.float32)
    y = torch.empty((rows, 2), dtype=torch.float32, device="cuda")
    lap_mlp_forward(torch.tensor(packed(p), dtype=torch.float32, device="cuda"), torch.from_numpy(x).cuda(), rows, y)
    pf = {k: np.float32(v).astype(np.float64) for k, v in p.items()}
    ref, cache = CV.forward(pf, x.astype(np.float64))
    got = y.cpu().numpy()
    # Every output within the element-wise bound, or (a few) within the
    # deviation that BF16 rounding decisions at FP32 precision allow.
    rms = np.sqrt(np.mean(ref * ref, axis=0, keepdims=True))
    err = np.abs(got - ref)
    tight = err <= 1e-2 * np.abs(ref) + 2e-3 * rms
    assert np.all(tight | (err <= rounding_bound(pf, cache))), np.argwhere(~tight)[:5]
    assert (~tight).mean() < 1e-4


def rounding_bound(pf, cache):
    """Largest deviation of an output of the FP32 kernel from the FP64 oracle
    that the shared BF16 rounding points allow.  Each FP32 sum (at most 65
    terms, bias included) is within e = 65 * 2^-22 * sum|terms| of the exact
    one (a 4x margin over round-to-nearest).  A hidden activation whose
    interval [z - d, z + d] (after the ReLU) spans two BF16 values may round
    to either on the GPU: u = that gap; layer 2's interval adds layer 1's
    gaps through |W2|, and the output deviates by its own FP32 error plus
    layer 2's gaps through |W3|."""
    xb, W1, W2, W3, z1, h1, z2, h2 = cache
    e = 65 * 2.0 ** -22
    d1 = e * (np.abs(xb) @ np.abs(W1).T + np.abs(pf["b1"]))
    u1 = np.abs(CV.bf16(np.maximum(z1 + d1, 0.0)) - CV.bf16(np.maximum(z1 - d1, 0.0)))
    d2 = e * (np.abs(h1) @ np.abs(W2).T + np.abs(pf["b2"])) + u1 @ np.abs(W2).T
    u2 = np.abs(CV.bf16(np.maximum(z2 + d2, 0.0)) - CV.bf16(np.maximum(z2 - d2, 0.0)))
    return e * (np.abs(h2) @ np.abs(W3).T + np.abs(pf["b3"])) + u2 @ np.abs(W3).T


def relu_fixed_rows(pf, x):
    """Rows on which every ReLU decision (the sign of a pre-activation) is
    fixed by the arithmetic: |z| exceeds the FP32 error bound of its sum (as
    in rounding_bound, layer 2 including layer 1's BF16 rounding gaps).  On
    other rows the FP32 kernel may zero a back-propagated error that the
    FP64 oracle keeps, or the reverse."""
    _, (xb, W1, W2, _, z1, h1, z2, _) = CV.forward(pf, np.asarray(x, dtype=np.float64))
    e = 65 * 2.0 ** -22
    d1 = e * (np.abs(xb) @ np.abs(W1).T + np.abs(pf["b1"]))
    u1 = np.abs(CV.bf16(np.maximum(z1 + d1, 0.0)) - CV.bf16(np.maximum(z1 - d1, 0.0)))
    d2 = e * (np.abs(h1) @ np.abs(W2).T + np.abs(pf["b2"])) + u1 @ np.abs(W2).T
    return np.all(np.abs(z1) > d1, axis=1) & np.all(np.abs(z2) > d2, axis=1)


@pytest.mark.parametrize("rows", [37, 128, 640, 5003, 40_000])
def test_mlp_loss_and_gradients_match_oracle(rows, mlp_kernel):
    """40,000 rows are 313 tiles of 128: more tiles than CTAs, so the weight
    gradients accumulate over several tiles per CTA."""
    p = _params(3)
    pf = {k: np.float32(v).astype(np.float64) for k, v in p.items()}
    rng = np.random.default_rng(4)
    x = rng.standard_normal((rows + rows // 10 + 8, 8)).astype(np.float32)
    x = x[relu_fixed_rows(pf, x)][:rows]
    assert x.shape[0] == rows
    t = rng.standard_normal((rows, 2)).astype(np.float32)
    grad = torch.zeros(LAP_MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    lap_mlp_loss_grad(torch.tensor(packed(p), dtype=torch.float32, device="cuda"), torch.from_numpy(x).cuda(),
                      torch.from_numpy(t).cuda(), rows, 1.0, 0.5, grad, loss)
    lo, go = CV.loss_and_grads(pf, x.astype(np.float64), t.astype(np.float64), w=(1.0, 0.5))
    assert loss.item() == pytest.approx(lo, rel=1e-3)
    g = unpack(grad.cpu().numpy())
    for k in go:
        assert_elementwise(g[k], go[k], axis=None, what=k)


def test_adamw_matches_oracle():
    rng = np.random.default_rng(6)
    w = rng.standard_normal(LAP_MLP_PARAMS).astype(np.float32)
    m = np.zeros_like(w)
    v = np.zeros_like(w)
    W, M, V = (torch.from_numpy(a.copy()).cuda() for a in (w, m, v))
    wo, mo, vo = w.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for step in range(1, 6):
        g = rng.standard_normal(LAP_MLP_PARAMS).astype(np.float32)
        lap_adamw(W, M, V, torch.from_numpy(g).cuda(), LAP_MLP_PARAMS, step, 1e-2, weight_decay=0.01)
        wo, mo, vo = CV.adamw_step(wo, mo, vo, g.astype(np.float64), step, 1e-2, wd=0.01)
    np.testing.assert_allclose(W.cpu().numpy(), wo, rtol=1e-5, atol=1e-6)


def test_trained_network_reduces_kemeny_variance():
    """Train on sampler-produced targets of 10 generated graphs, apply to a
    held-out Barabasi-Albert graph: the pi-walk control variate with the
    network's hitting-time potential must cut the per-sample variance of
    Y1 - Y2 (the Kemeny estimator) by at least 20% on fresh samples, and the
    CV estimate must stay consistent with the dense Kemeny constant."""
    sets = []
    for k in range(10):
        g = I.ba(int(2000 + 700 * k), 2 + k % 4, seed=100 + k) if k % 2 == 0 else I.rmat(11 + k % 2, 6, seed=100 + k)
        G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 28)
        G.set_root()
        sets.append(CVG.training_targets(G, omega=256, reps=8, seed=10 + k))
        G.close()
    params, hist = CVG.train(sets, epochs=6, batch=4096)
    assert hist[-1] < hist[0]
    g = I.ba(1500, 3, seed=999)
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 28)
    try:
        G.set_root()
        phi1, phi2 = CVG.pilot_potentials(G, params, seed=5, samples=1024)
        beta1, beta2 = CVG.fit_betas(G, phi1, phi2, seed=77, pilot=4096)
        a, b, m = G.sample_trace_cv(8192, 5)
        est = (a - b).double().cpu().numpy()
        cv = est + beta2 * m.cpu().numpy()
        _, _, kc_cv, _ = G.cv_estimates(beta1, beta2)
    finally:
        G.close()
    ratio = np.var(cv) / np.var(est)
    assert ratio < 0.8, ratio
    kc = D.kemeny(g.n, g.row_ptr, g.col)
    se = np.std(cv) / np.sqrt(cv.size)
    assert abs(kc_cv - kc) < 6 * se, (kc_cv, kc, se)


def test_cv_targets_match_oracle():
    """lap_cv_targets: FP64 ratios of the handle's counts and of fresh
    hitting walks, rounded to float32: bit-exact with the oracle's statement
    on the same counts and walks."""
    g = I.ba(3000, 3, seed=12)
    omega, reps, seed = 200, 6, 41
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 26)
    try:
        v = G.set_root()
        G.sample(omega, seed)
        t = G.cv_targets(reps, seed + 1).cpu().numpy()
    finally:
        G.close()
    c = oracle.sample(g.row_ptr, g.col, v, seed, 0, omega)
    hit = oracle.hitting_walks(g.row_ptr, g.col, v, seed + 1, reps)
    want = CV.training_targets(c.cnt1, omega, hit, reps, c.sum_y2, v)
    assert np.array_equal(t, want)


def test_cv_potentials_match_oracle():
    """lap_cv_potentials: phi1 = y0 / d, phi2 = y1 * (sum Y2 / omega) of the
    samples drawn, phi2(v) = 0: bit-exact with the oracle's statement."""
    g = I.er(500, 0.02, seed=8)
    rng = np.random.default_rng(9)
    y = rng.uniform(0.1, 5.0, (g.n, 2)).astype(np.float32)
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 24)
    try:
        v = G.set_root()
        G.sample(300, 2)
        phi1, phi2 = G.cv_potentials(torch.from_numpy(y).cuda())
        _, _, sums = G.counts()
    finally:
        G.close()
    w1, w2 = CV.potentials(y, g.row_ptr, v, float(sums[2]) / 300.0)
    assert np.array_equal(phi1.cpu().numpy(), w1) and np.array_equal(phi2.cpu().numpy(), w2)


@pytest.mark.parametrize("kernel", [1, 2], ids=["wide", "compact"])
def test_cv_fit_betas_match_oracle(kernel):
    """lap_cv_fit_betas draws the pilot batches on the GPU and reduces them
    there; its per-batch integers equal the oracle's bit for bit, so the
    coefficients differ only by the order of FP64 sums (1e-9 relative).  The
    handle is left as after lap_set_root: the next samples start at id 0."""
    g = I.ba(3000, 3, seed=13)
    rng = np.random.default_rng(14)
    phi1 = rng.uniform(0.0, 2.0, g.n)
    phi2 = rng.uniform(0.0, 40.0, g.n)
    first, per, batches, seed = (1 << 31) + 5, 150, 6, 21
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 26)
    try:
        G.set_option(LAP_OPT_KERNEL, kernel)
        v = G.set_root()
        b1, b2 = G.cv_fit_betas(torch.from_numpy(phi1).cuda(), torch.from_numpy(phi2).cuda(), seed, first,
                                per * batches, batches)
        G.sample(20, 3)
        c1, _, s = G.counts()
    finally:
        G.close()
    w1, w2 = CV.fit_betas(g.row_ptr, g.col, v, seed, first, per, batches, CV.quantize_potential(phi1),
                          CV.quantize_potential(phi2))
    assert b1 == pytest.approx(w1, rel=1e-9) and b2 == pytest.approx(w2, rel=1e-9)
    assert b1 != 0.0 and b2 != 0.0
    c = oracle.sample(g.row_ptr, g.col, v, 3, 0, 20)
    assert int(s[0]) == 20 and np.array_equal(c1, c.cnt1)


def test_cv_sums_merge_across_handles():
    """Two handles draw disjoint sample-id ranges with the same potentials;
    their integer counts and control-variate sums, added on the host and
    loaded into a third handle (lap_set_counts, then lap_cv_set_sums), give
    the control-variate estimates of one handle that drew every id, bit for
    bit."""
    from paper_2311_10290_gb300.lap import LAP_OPT_CURSOR
    g = I.ba(2500, 3, seed=21)
    rng = np.random.default_rng(22)
    phi1 = torch.from_numpy(rng.uniform(0.0, 2.0, g.n)).cuda()
    phi2 = torch.from_numpy(rng.uniform(0.0, 30.0, g.n)).cuda()

    def run(first, count):
        G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 26)
        G.set_root()
        G.set_option(LAP_OPT_CURSOR, first)
        G.cv_set_potentials(phi1, phi2)
        G.sample(count, 8)
        return G

    whole = run(0, 500)
    a, b = run(0, 180), run(180, 320)
    try:
        ca, cb = a.counts(), b.counts()
        sa, sb = a.cv_sums(), b.cv_sums()
        m = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 22)
        m.set_root()
        m.cv_set_potentials(phi1, phi2)
        m.set_counts(ca[0] + cb[0], ca[1] + cb[1], (ca[2] + cb[2])[:3])
        m.cv_set_sums(*(x + y for x, y in zip(sa, sb)))
        got = m.cv_estimates(0.7, 1.3)
        want = whole.cv_estimates(0.7, 1.3)
        m.close()
    finally:
        for G in (whole, a, b):
            G.close()
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    assert got[2] == want[2] and got[3] == want[3]
