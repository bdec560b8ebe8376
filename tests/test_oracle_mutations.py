"""The oracle's pins catch plausible mistakes: each case plants one mistake
(a dropped term or factor, a wrong sign or index, a wrong Philox key word, a
start drawn from the wrong law, a visit not counted, an eigenvalue dropped
from the dense truth, the SpanTree subtree test the other way round) in a
copy of the oracle outside the repository and runs the pins of that part
(tests/test_oracle_pins.py for the LEWalk sampler, finalize and dense truth,
tests/test_oracle_cv_pins.py for the control variate,
tests/test_oracle_spantree_pins.py for Alg. 1 / Alg. 3 and
tests/test_oracle_cg_pins.py for the sparse solves) against the copy; at
least one pin must fail.  The repository's oracle is not
touched."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_PINS = "test_oracle_pins.py"
ST_PINS = "test_oracle_spantree_pins.py"
CV_PINS = "test_oracle_cv_pins.py"
CG_PINS = "test_oracle_cg_pins.py"

# (name, file under oracle/, anchor, planted mistake, pins that must catch it)
MUTATIONS = [
    ("ldiag_factor_2_dropped", "lewalk_oracle.c",
     "ld[u] = (u == v) ? lvv : (y1[u] - 2.0 * y2[u]) + lvv;",
     "ld[u] = (u == v) ? lvv : (y1[u] - 1.0 * y2[u]) + lvv;", C_PINS),
    ("retrace_skips_the_start", "lewalk_oracle.c",
     "        u = s;\n        while (!intree[u]) {\n            intree[u] = 1;",
     "        u = next[s];\n        while (u >= 0 && !intree[u]) {\n            intree[u] = 1;", C_PINS),
    ("stack_index_not_advanced", "lewalk_oracle.c",
     "            draws[u] += 1;\n            next[u] = oracle_neighbor",
     "            draws[u] += (u & 1);\n            next[u] = oracle_neighbor", C_PINS),
    ("walk_start_not_counted", "lewalk_oracle.c",
     "            cnt2[u] += 1;\n            t += 1;",
     "            t += 1;\n            if (t > 1) cnt2[u] += 1;", C_PINS),
    ("pi_start_drawn_uniformly", "lewalk_oracle.c",
     "int32_t u = col[oracle_below(oracle_r64(seed, 0u, 0u, i, 2u), (uint64_t)arcs)];",
     "int32_t u = (int32_t)oracle_below(oracle_r64(seed, 0u, 0u, i, 2u), (uint64_t)n);", C_PINS),
    ("ecc_extra_term", "lewalk_oracle.c",
     "ecc[u] = (double)(n - 1) / ((double)n * ld[u] + tr);",
     "ecc[u] = (double)(n - 1) / ((double)n * ld[u] + tr - lvv);", C_PINS),
    ("lvv_divided_twice", "lewalk_oracle.c",
     "    double lvv = s2 / (double)n;",
     "    double lvv = s2 / (double)n / (double)n;", C_PINS),
    ("philox_wrong_key_word", "lewalk_oracle.c",
     "y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;",
     "y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k1;", C_PINS),
    ("first_visit_not_counted", "lewalk_oracle.c",
     "            cnt1[u] += 1;\n            y1 += 1;",
     "            y1 += 1;\n            if (draws[u]) cnt1[u] += 1;", C_PINS),
    ("kemeny_sign", "lewalk_oracle.c",
     "*kemeny = ((double)sum_y1 - (double)sum_y2) / w;",
     "*kemeny = ((double)sum_y1 + (double)sum_y2) / w;", C_PINS),
    ("y2_not_divided_by_degree", "lewalk_oracle.c",
     "y2[u] = (double)cnt2[u] / (w * d);",
     "y2[u] = (double)cnt2[u] / w;", C_PINS),
    ("path_departure_not_advanced", "lewalk_oracle.c",
     "                draws[u] += 1;\n                u = oracle_neighbor(row_ptr, col, u, x);",
     "                draws[u] += (u & 1);\n                u = oracle_neighbor(row_ptr, col, u, x);", C_PINS),
    ("pinv_drops_an_eigenvalue", "dense.py",
     "    inv[1:] = 1.0 / lam[1:]",
     "    inv[2:] = 1.0 / lam[2:]", C_PINS),
    ("ecc_trace_dropped", "dense.py",
     "    return (n - 1) / (n * dg + dg.sum())",
     "    return (n - 1) / (n * dg)", C_PINS),
    ("kemeny_drops_an_eigenvalue", "dense.py",
     "    return float(np.sum(1.0 / sig[1:]))",
     "    return float(np.sum(1.0 / sig[2:]))", C_PINS),
    ("rwb_missing_factor_n", "dense.py",
     "    return tr, 1.0 / n + tr / ((n - 1) * (tr + n * ld))",
     "    return tr, 1.0 / n + tr / ((n - 1) * (tr + ld))", C_PINS),
    ("cv_draw_potential_of_the_wrong_node", "lewalk_oracle.c",
     "if (cv && cv->h1) cv->a1[u] += cv->h1[next[u]];",
     "if (cv && cv->h1) cv->a1[u] += cv->h1[u];", CV_PINS),
    ("cv_pi_martingale_sign", "lewalk_oracle.c",
     "m2 += (double)(d * cv->h2[w] - cv->S2[u]) / (double)d;",
     "m2 += (double)(cv->S2[u] - d * cv->h2[w]) / (double)d;", CV_PINS),
    ("hitting_walk_last_step_dropped", "lewalk_oracle.c",
     "            sums[u] += t;",
     "            sums[u] += t - 1;", CV_PINS),
    ("bf16_ties_away_from_even", "cv.py",
     "    rounded = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16",
     "    rounded = ((b + 0x8000) >> 16) << 16", CV_PINS),
    ("relu_derivative_dropped", "cv.py",
     "    dh2 = (dyq @ W3) * (z2 > 0)",
     "    dh2 = (dyq @ W3)", CV_PINS),
    ("bf16_backward_rounding_point_moved", "cv.py",
     """    g = {"W3": dyq.T @ h2, "b3": dy.sum(axis=0)}""",
     """    g = {"W3": dy.T @ h2, "b3": dyq.sum(axis=0)}""", CV_PINS),
    ("adamw_second_moment_not_corrected", "cv.py",
     "    vh = v / (1.0 - beta2 ** step)",
     "    vh = v", CV_PINS),
    ("martingale_z1_sign", "cv.py",
     "    return d * np.asarray(a1, dtype=np.int64) - np.asarray(cnt1, dtype=np.int64) * s1",
     "    return d * np.asarray(a1, dtype=np.int64) + np.asarray(cnt1, dtype=np.int64) * s1", CV_PINS),
    ("beta1_variate_not_centred", "cv.py",
     "    Zc = Z - Z.mean(axis=0)",
     "    Zc = Z", CV_PINS),
    ("beta2_sign", "cv.py",
     "    beta2 = -float(c[0, 1]) / float(c[1, 1]) if c[1, 1] > 0 else 0.0",
     "    beta2 = float(c[0, 1]) / float(c[1, 1]) if c[1, 1] > 0 else 0.0", CV_PINS),
    ("hitting_target_not_divided_by_reps", "cv.py",
     "    t[:, 1] = (hit / float(reps)) / mean_y2",
     "    t[:, 1] = hit / mean_y2", CV_PINS),
    ("cv_kemeny_term_sign", "cv.py",
     "    kc = ((float(sum_y1) - float(sum_y2)) + beta2 * m2) / w",
     "    kc = ((float(sum_y1) - float(sum_y2)) - beta2 * m2) / w", CV_PINS),
    ("subtree_test_printed_direction", "spantree.py",
     "                if inside(u, e1):",
     "                if inside(e1, u):", ST_PINS),
    ("x2_sign_of_reversed_edge", "spantree.py",
     "                x2[u] -= size[e2]",
     "                x2[u] += size[e2]", ST_PINS),
    ("x2d_size_for_degree_sum", "spantree.py",
     "                x2d[u] += dsum[e1]",
     "                x2d[u] += size[e1]", ST_PINS),
    ("spantree_ldiag_factor_2_dropped", "spantree.py",
     "    ld = x1 - 2.0 * x2 + mean_x2",
     "    ld = x1 - x2 + mean_x2", ST_PINS),
    ("spantree_kemeny_sign", "spantree.py",
     "    return ld, ecc, t1 - t2",
     "    return ld, ecc, t1 + t2", ST_PINS),
    ("cg_residual_update_uses_the_direction", "cg.py",
     "        r -= alpha * q",
     "        r -= alpha * p", CG_PINS),
    ("cg_uniform_target_not_divided_by_n", "cg.py",
     "    y2 = r1 / n",
     "    y2 = r1", CG_PINS),
]


def run_pins_on_copy(tmp_path, fname, src, pins):
    """Runs the pins file `pins` against a copy of oracle/ whose `fname` holds
    `src`; returns pytest's exit code (0 all passed, 1 some failed)."""
    copy = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), copy,
                    ignore=shutil.ignore_patterns("*.so", "*.so.tmp*", "__pycache__"))
    (copy / fname).write_text(src)
    env = dict(os.environ)
    env["PYTHONPATH"] = os.pathsep.join([str(tmp_path), ROOT] + ([env["PYTHONPATH"]] if env.get("PYTHONPATH") else []))
    # Run from the copy's parent so that `import oracle` finds the copy first;
    # the pins and the input generators come from the repository.
    r = subprocess.run([sys.executable, "-c",
                        "import oracle, sys; assert oracle.__file__.startswith(sys.argv[1]), oracle.__file__",
                        str(tmp_path)], cwd=tmp_path, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-1000:]
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pins),
                        "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu"],
                       cwd=tmp_path, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, r.stdout


@pytest.mark.slow
@pytest.mark.parametrize("fname,pins", [("lewalk_oracle.c", C_PINS), ("dense.py", C_PINS), ("cv.py", CV_PINS),
                                        ("spantree.py", ST_PINS), ("cg.py", CG_PINS)])
def test_unchanged_copy_passes_the_pins(fname, pins, tmp_path):
    src = open(os.path.join(ROOT, "oracle", fname)).read()
    code, out = run_pins_on_copy(tmp_path, fname, src, pins)
    assert code == 0, out[-2000:]


@pytest.mark.slow
@pytest.mark.parametrize("name,fname,anchor,planted,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(name, fname, anchor, planted, pins, tmp_path):
    src = open(os.path.join(ROOT, "oracle", fname)).read()
    assert src.count(anchor) == 1, "mutation anchor not found once: %s" % name
    code, out = run_pins_on_copy(tmp_path, fname, src.replace(anchor, planted), pins)
    assert code == 1, "no pin failed with the planted mistake %s:\n%s" % (name, out[-2000:])
