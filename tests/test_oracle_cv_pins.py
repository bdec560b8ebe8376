"""Pins for the control-variate oracle (oracle/cv.py and oracle_sample_cv):
BF16 rounding, MLP gradients (finite differences), AdamW, features on hand
checked graphs, the zero-mean identity of the martingale increments, and the
variance cancellation the hitting-time potential must produce.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import oracle.cv as CV
import oracle.dense as D
from paper_2311_10290_gb300 import inputs as I


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.0e-3, 65504.0, 1.0 + 2 ** -7])
    want = np.array([1.0, 1.0, 1.0 + 2 ** -7, -2.5, None, None, 1.0 + 2 ** -7], dtype=object)
    got = CV.bf16(x)
    for g, w in zip(got, want):
        if w is not None:
            assert g == w
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(0).standard_normal(10000) * 10
    ref = torch.from_numpy(r.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(CV.bf16(r), ref)


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    p = CV.init_params(3)
    for k in p:
        p[k] = p[k] + 0.05 * rng.standard_normal(p[k].shape)
    x = rng.standard_normal((37, CV.N_FEAT))
    t = rng.standard_normal((37, CV.N_OUT))
    loss, g = CV.loss_and_grads(p, x, t, w=(1.0, 0.5), quantize=False)
    eps = 1e-6
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _ = CV.loss_and_grads(p, x, t, w=(1.0, 0.5), quantize=False)
            flat[idx] = old - eps
            lm, _ = CV.loss_and_grads(p, x, t, w=(1.0, 0.5), quantize=False)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, an)


def test_bf16_training_reduces_to_the_exact_gradients_on_bf16_values():
    """With inputs, weights, targets and every intermediate exactly
    representable in BF16 (small dyadic values), the BF16 statement of the
    backward pass equals the exact one, which the finite-difference pin
    fixes."""
    rng = np.random.default_rng(4)
    H, F, O = CV.HIDDEN, CV.N_FEAT, CV.N_OUT

    def sparse(rows, cols, per_row):
        """Entries +-1/2, `per_row` per row; with per_row = 2 and rows = cols,
        two per column too (two permutations), so every product has at most
        two nonzero terms and stays a short dyadic number."""
        m = np.zeros((rows, cols))
        for k in range(per_row):
            perm = rng.permutation(max(rows, cols))[:rows] % cols if rows != cols else rng.permutation(cols)
            m[np.arange(rows), perm] = rng.choice([-0.5, 0.5], rows)
        return m

    p = {"W1": sparse(H, F, 1), "b1": rng.choice([-0.5, 0.0, 0.5], H),
         "W2": sparse(H, H, 2), "b2": rng.choice([-0.5, 0.0, 0.5], H),
         "W3": sparse(O, H, 2), "b3": np.array([0.5, -0.25])}
    x = rng.integers(-1, 2, (4, F)).astype(np.float64)
    t = rng.integers(-4, 5, (4, O)) / 2.0
    lq, gq = CV.loss_and_grads(p, x, t, w=(1.0, 0.5), quantize=True)
    le, ge = CV.loss_and_grads(p, x, t, w=(1.0, 0.5), quantize=False)
    assert lq == le
    for k in ge:
        assert np.array_equal(gq[k], ge[k]), k


def test_bf16_backward_rounds_the_output_error_only_where_it_enters_a_product():
    """One row, one hidden unit active, y - t chosen so that dY = 1 + 2^-10
    (not a BF16 value: it rounds to 1): the W3 gradient takes the rounded
    dY (1 * h2), the b3 gradient the unrounded one."""
    p = {"W1": np.zeros((CV.HIDDEN, CV.N_FEAT)), "b1": np.zeros(CV.HIDDEN),
         "W2": np.zeros((CV.HIDDEN, CV.HIDDEN)), "b2": np.zeros(CV.HIDDEN),
         "W3": np.zeros((CV.N_OUT, CV.HIDDEN)), "b3": np.zeros(CV.N_OUT)}
    p["b1"][0] = 1.0
    p["W2"][0, 0] = 1.0           # h1[0] = 1, h2[0] = 1, every other unit 0
    x = np.zeros((1, CV.N_FEAT))
    t = np.array([[-(1.0 + 2.0 ** -10) / 2.0, 0.0]])     # y = 0, dY0 = 2 (y - t) = 1 + 2^-10
    _, g = CV.loss_and_grads(p, x, t, w=(1.0, 1.0), quantize=True)
    assert g["b3"][0] == 1.0 + 2.0 ** -10
    assert g["W3"][0, 0] == 1.0
    _, ge = CV.loss_and_grads(p, x, t, w=(1.0, 1.0), quantize=False)
    assert ge["W3"][0, 0] == 1.0 + 2.0 ** -10


def test_adamw_first_step_closed_form():
    w = np.array([0.5, -1.0, 2.0])
    g = np.array([0.3, -0.001, 0.0])
    w1, m, v = CV.adamw_step(w, np.zeros(3), np.zeros(3), g, 1, lr=0.01, wd=0.1, eps=1e-8)
    # first step: m_hat = g, v_hat = g^2, so the step is lr*(g/(|g|+eps) + wd*w)
    want = w - 0.01 * (g / (np.abs(g) + 1e-8) + 0.1 * w)
    assert np.allclose(w1, want, rtol=1e-12, atol=1e-15)


def test_features_on_a_path_rooted_at_an_end():
    g = I.path(5)                      # 0-1-2-3-4, root 0
    f = CV.features(g.row_ptr, g.col, 0)
    d = np.array([1, 2, 2, 2, 1.0])
    assert np.allclose(f[:, 0], np.log(d)) and np.allclose(f[:, 1], 1 / d)
    assert np.allclose(f[:, 2], np.log1p([0, 1, 2, 3, 4]))
    assert np.array_equal(f[:, 3], [0, 1, 0, 0, 0])
    assert np.allclose(f[:, 4], np.log([2, 1.5, 2, 1.5, 2]))      # mean neighbour degree
    assert np.allclose(f[:, 5], [0, 0.5, 0, 0.5, 0.0])            # share of degree-1 neighbours (nodes 0, 4)
    # two-hop degree sums: s1 = [2,3,4,3,2]; s2 = [3,6,6,6,3]
    assert np.allclose(f[:, 6], np.log(np.array([3, 6, 6, 6, 3.0]) / np.array([2, 3, 4, 3, 2.0])))
    # P(hit 0 within 8 steps): node 1 -> 1/2 + 1/4*... computed by brute force on the chain
    P = np.zeros((5, 5))
    for u in range(1, 5):
        for w in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]:
            P[u, w] = 1 / d[u]
    P[0, 0] = 1.0
    hit = np.linalg.matrix_power(P, 8)[:, 0]
    assert np.allclose(f[:, 7], hit)


def test_martingale_increments_sum_to_zero_over_neighbours():
    g = I.ba(300, 3, seed=2)
    h = np.random.default_rng(0).integers(-2 ** 30, 2 ** 30, size=g.n)
    s = CV.neighbour_sums(g.row_ptr, g.col, h)
    for u in range(g.n):
        nb = g.col[g.row_ptr[u]:g.row_ptr[u + 1]]
        assert int(np.sum(len(nb) * h[nb] - s[u])) == 0


def test_constant_potential_gives_zero_terms_and_plain_estimates():
    g = I.er(200, 0.04, seed=3)
    v = oracle.root_max_degree(g.row_ptr)
    c = np.full(g.n, 12345, dtype=np.int64)
    cnt, a1, a2, p2, m2 = oracle.sample_cv(g.row_ptr, g.col, v, 9, 0, 300, h1=c, h2=c)
    z1 = CV.martingale_z1(g.row_ptr, g.col, c, cnt.cnt1, a1)
    assert np.all(z1 == 0) and np.all(m2 == 0.0)
    assert CV.martingale_m2(g.row_ptr, g.col, c, a2, p2) == 0.0
    plain = oracle.sample(g.row_ptr, g.col, v, 9, 0, 300)
    assert np.array_equal(plain.cnt1, cnt.cnt1) and np.array_equal(plain.cnt2, cnt.cnt2)
    ld0, ec0, kc0 = oracle.finalize(g.row_ptr, v, 300, cnt.cnt1, cnt.cnt2, cnt.sum_y1, cnt.sum_y2)
    ld1, ec1, kc1 = CV.finalize_cv(g.row_ptr, v, 300, cnt.cnt1, cnt.cnt2, cnt.sum_y1, cnt.sum_y2, z1, 0.0, 0.7, 0.9)
    assert np.allclose(ld0, ld1, rtol=1e-13) and np.allclose(ec0, ec1, rtol=1e-13) and kc0 == pytest.approx(kc1, rel=1e-14)


def test_per_sample_m2_adds_up_to_the_node_totals():
    g = I.ba(500, 2, seed=5)
    v = oracle.root_max_degree(g.row_ptr)
    h2 = np.random.default_rng(1).integers(0, 2 ** 26, size=g.n)
    cnt, a1, a2, p2, m2 = oracle.sample_cv(g.row_ptr, g.col, v, 4, 0, 400, h2=h2)
    total = CV.martingale_m2(g.row_ptr, g.col, h2, a2, p2)
    assert math.fsum(m2.tolist()) == pytest.approx(total, rel=1e-9, abs=1e-3)
    assert int(p2.sum()) == cnt.sum_y2          # one pi-walk step per pass before absorption


def test_martingale_terms_have_mean_zero():
    g = I.rmat(8, 6, seed=4)
    v = oracle.root_max_degree(g.row_ptr)
    rng = np.random.default_rng(2)
    h = rng.integers(0, 2 ** 24, size=g.n)
    zs, ms = [], []
    for b in range(30):
        cnt, a1, a2, p2, m2 = oracle.sample_cv(g.row_ptr, g.col, v, 11, 500 * b, 500, h1=h, h2=h)
        zs.append(CV.martingale_z1(g.row_ptr, g.col, h, cnt.cnt1, a1).sum() / 2 ** 24 / 500)
        ms.append(m2.sum() / 2 ** 24 / 500)
    for x in (np.array(zs), np.array(ms)):
        assert abs(x.mean()) < 6 * x.std(ddof=1) / np.sqrt(len(x))


def test_hitting_time_potential_cancels_the_pi_walk_variance():
    """With h2 = hitting time h(., v), Y2 - M2 = h(start, v): the walk's own
    randomness cancels, so its variance drops to that of the start's hitting
    time (here below 10% of Var(Y2)); a sign or index error breaks this."""
    g = I.ba(400, 2, seed=7)
    v = oracle.root_max_degree(g.row_ptr)
    hit = D.hitting_times_to(g.n, g.row_ptr, g.col, v)
    h2 = CV.quantize_potential(hit)
    cnt, a1, a2, p2, m2 = oracle.sample_cv(g.row_ptr, g.col, v, 3, 0, 4000, h2=h2)
    y2 = cnt.y2.astype(np.float64)
    resid = y2 - m2 / 2.0 ** CV.FIXED_POINT_BITS
    pi = g.degree / g.degree.sum()
    var_start = float(pi @ hit ** 2 - (pi @ hit) ** 2)
    assert np.var(resid) < 0.1 * np.var(y2)
    assert np.var(resid) == pytest.approx(var_start, rel=0.2)


def test_cv_kemeny_estimate_with_the_hitting_time_potential():
    """finalize_cv's Kemeny estimate (ΣY1 − ΣY2 + β2 M2)/ω with h2 = the
    hitting time h(., v) and β2 = 2^-16 (one unit of the fixed-point
    potential): every π walk's own randomness cancels, leaving its start's
    hitting time, and E[M2] = 0 keeps the estimate unbiased.  Across 300
    batches of 10 samples the estimates stay within 6 standard errors of the
    dense κ and vary less than 0.8 times as much as the plain estimates of the
    same samples (about 0.5 on this graph; the opposite sign of the term
    doubles the walk's randomness instead: about 2.5)."""
    g = I.er(200, 0.03, seed=3)
    v = oracle.root_max_degree(g.row_ptr)
    hit = D.hitting_times_to(g.n, g.row_ptr, g.col, v)
    h2 = CV.quantize_potential(hit)
    z1 = np.zeros(g.n, dtype=np.int64)
    beta2 = 2.0 ** -CV.FIXED_POINT_BITS
    kc_t = D.kemeny(g.n, g.row_ptr, g.col)
    plain, cv = [], []
    for b in range(300):
        cnt, a1, a2, p2, m2 = oracle.sample_cv(g.row_ptr, g.col, v, 5, 10 * b, 10, h2=h2)
        m2_total = CV.martingale_m2(g.row_ptr, g.col, h2, a2, p2)
        plain.append(oracle.finalize(g.row_ptr, v, 10, cnt.cnt1, cnt.cnt2, cnt.sum_y1, cnt.sum_y2)[2])
        cv.append(CV.finalize_cv(g.row_ptr, v, 10, cnt.cnt1, cnt.cnt2, cnt.sum_y1, cnt.sum_y2, z1, m2_total,
                                 0.0, beta2)[2])
    plain, cv = np.array(plain), np.array(cv)
    assert np.var(cv) < 0.8 * np.var(plain), (np.var(cv), np.var(plain))
    assert abs(cv.mean() - kc_t) < 6 * cv.std(ddof=1) / np.sqrt(len(cv))
    assert abs(plain.mean() - kc_t) < 6 * plain.std(ddof=1) / np.sqrt(len(plain))


def test_hitting_walks_estimate_the_hitting_times():
    """The control variate's hitting-time targets (Section 3.2, v-absorbed
    walk lemma: E[length of a walk from u absorbed at v] = h(u, v) =
    (L_v^{-1} d)_u): batch means of the oracle's walk lengths fall within 6
    standard errors of the dense h(., v) at every node; on a star rooted at
    its hub every walk from a leaf is exactly one step."""
    g = I.ba(120, 2, seed=11)
    v = oracle.root_max_degree(g.row_ptr)
    hit = D.hitting_times_to(g.n, g.row_ptr, g.col, v)
    reps = 40
    batches = np.array([oracle.hitting_walks(g.row_ptr, g.col, v, 1000 + b, reps).astype(np.float64) / reps
                        for b in range(25)])
    mean, se = batches.mean(axis=0), batches.std(axis=0, ddof=1) / np.sqrt(len(batches))
    keep = np.arange(g.n) != v
    assert np.all(np.abs(mean - hit)[keep] <= 6 * se[keep] + 1e-9)
    assert np.all(batches[:, v] == 0.0)
    s = I.star(30)
    sums = oracle.hitting_walks(s.row_ptr, s.col, 0, 5, 7)
    assert sums[0] == 0 and np.all(sums[1:] == 7)


def test_betas_recover_exact_linear_relations():
    """Noise-free data on a line: V = c_u + 2.5 Z (an offset per node, which
    the per-node centring removes) gives beta1 = 2.5; y = 7 - 1.5 m gives
    beta2 = 1.5 (the Kemeny variate enters as + beta2 m).  Constant Z or m
    give 0."""
    rng = np.random.default_rng(3)
    Z = rng.standard_normal((6, 40))
    V = rng.uniform(0, 100, 40)[None, :] + 2.5 * Z
    m = rng.standard_normal(500)
    y = 7.0 - 1.5 * m
    b1, b2 = CV.betas_from_batches(V, Z, y, m)
    assert b1 == pytest.approx(2.5, rel=1e-13) and b2 == pytest.approx(1.5, rel=1e-13)
    b1, b2 = CV.betas_from_batches(V, np.ones((6, 40)), y, np.full(500, 3.0))
    assert b1 == 0.0 and b2 == 0.0


def test_fitted_beta2_with_the_hitting_time_potential_is_one_unit():
    """With h2 = round(2^16 h(., v)), Y2 - 2^-16 M2 is the start's hitting
    time, and the visits of the (independent) Wilson run do not depend on
    M2, so the least-squares beta2 is 2^-16 (one unit of the fixed-point
    potential) up to sampling error (about 0.5% here)."""
    g = I.ba(400, 2, seed=7)
    v = oracle.root_max_degree(g.row_ptr)
    h2 = CV.quantize_potential(D.hitting_times_to(g.n, g.row_ptr, g.col, v))
    h1 = np.random.default_rng(0).integers(0, 2 ** 16, size=g.n)
    b1, b2 = CV.fit_betas(g.row_ptr, g.col, v, 5, 1 << 20, 500, 8, h1, h2)
    assert b2 * 2.0 ** CV.FIXED_POINT_BITS == pytest.approx(1.0, abs=0.05)
    assert np.isfinite(b1)


def test_targets_and_potentials_on_exact_expectations_give_the_estimands():
    """Fed the exact expectations (visits d_u (L_v^{-1})_uu per sample,
    hitting times h(u, v) per walk, E[Y2] = (1/2m) d^T L_v^{-1} d per
    sample), the targets are d_u (L_v^{-1})_uu and h(u, v) / E[Y2], and the
    potentials made from them with scale E[Y2] are (L_v^{-1})_uu and h(u, v)
    (float32 rounding of the targets: 1e-7)."""
    g = I.er(30, 0.2, seed=1)
    v = oracle.root_max_degree(g.row_ptr)
    e = D.expectations(g.n, g.row_ptr, g.col, v)
    hit = D.hitting_times_to(g.n, g.row_ptr, g.col, v)
    omega, reps = 1000, 16
    t = CV.training_targets(e["visits"] * omega, omega, hit * reps, reps, e["y2"] * omega, v)
    lv = D.lv_inverse(g.n, g.row_ptr, g.col, v)
    d = g.degree.astype(np.float64)
    keep = np.arange(g.n) != v
    np.testing.assert_allclose(t[keep, 0], (d * np.diag(lv))[keep], rtol=1e-6)
    np.testing.assert_allclose(t[keep, 1], (hit / e["y2"])[keep], rtol=1e-6)
    assert np.all(t[v] == 0.0)
    phi1, phi2 = CV.potentials(t, g.row_ptr, v, e["y2"])
    np.testing.assert_allclose(phi1[keep], np.diag(lv)[keep], rtol=1e-6)
    np.testing.assert_allclose(phi2, hit, rtol=1e-6, atol=0)
    assert phi2[v] == 0.0


def test_targets_on_a_hub_rooted_star_are_exact():
    """Rooted at the hub of a star, every leaf is visited exactly once per
    sample and every hitting walk from a leaf takes one step: t0 = 1 and
    t1 = 1 / (sum Y2 / omega) exactly."""
    g = I.star(40)
    omega, reps = 300, 4
    c = oracle.sample(g.row_ptr, g.col, 0, 3, 0, omega)
    hit = oracle.hitting_walks(g.row_ptr, g.col, 0, 4, reps)
    t = CV.training_targets(c.cnt1, omega, hit, reps, c.sum_y2, 0)
    assert np.all(t[1:, 0] == 1.0)
    assert np.all(t[1:, 1] == np.float32(1.0 / (c.sum_y2 / omega)))
    assert np.all(t[0] == 0.0)
