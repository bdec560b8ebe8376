#!/usr/bin/env python
"""Benchmark of the LEWalk hot path on GB300.

One "step" = one pass of the whole hot path over one batch of samples of the
workload graph: lap_sample (Wilson LE_v run + uniform-start and pi-start
v-absorbed walks per sample, counts folded into uint64 totals) followed by
the FP64 finalize (ECC for every node and Kemeny's constant).  The graph is
resident in HBM; graph ingest and root choice run once before timing.

Workload (default): Barabasi-Albert n = 10^6, m = 5, root = highest-degree
node; one step draws the workload's 2^16 samples (all in flight at once).

Printed: one JSON line (rank 0) with throughput in walk steps/s (Wilson steps
incl. loops + absorbed-walk steps), the sampler's HBM roofline, the CPU
oracle baseline, an end-to-end figure through the C ABI with host buffers,
clocks, and the time to reach relative error 1e-2 on the small Erdos-Renyi
workload against its dense FP64 ground truth.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# Algorithmic bytes per unit (32-byte sectors of random access):
#   Wilson step: row record, column entry, next node's state, state write,
#                visited test -> 5 sectors; tree insertion (retrace): state
#                read + write -> 2 sectors; absorbed-walk step: row record,
#                column entry, count -> 3 sectors.
SECTOR = 32
BYTES_WILSON_STEP = 5 * SECTOR
BYTES_TREE_INSERT = 2 * SECTOR
BYTES_WALK_STEP = 3 * SECTOR

# DRAM traffic per Wilson step (dram__bytes_read.sum + dram__bytes_write.sum of
# one sampler launch over the launch's Wilson steps, absorbed-walk steps and
# tree insertions included), from ncu captures of small cases of the same
# kernel and graph family (a 4 GB workspace, one launch; profiles/): the
# bench scales it by the Wilson steps of its own launch.  Valid only for the
# sources it was measured on (SHA-1 over the files listed).
TRAFFIC_PER_WILSON_STEP = {
    # 1-byte kernel, BA 10^6, 4096 samples in 3,535 lanes: 671.4 GB / 4.582e9 steps
    "lewalk_compact_kernel": (146.53, ("sampler_compact.cu", "compact_state.cuh", "philox.cuh"),
                              "98cf00da0b50c4c76b0ab9ce347f4a03af608187"),
    # several walkers, R-MAT scale 22, 2048 samples in 682 groups of 8: 623.8 GB / 4.986e9 steps
    "lewalk_group_kernel": (125.12, ("sampler_group.cu", "philox.cuh"), "fe1d23fff1727bcdef9d46436a9bcdcc51163c84"),
}


def sources_sha1(files):
    import hashlib
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_2311_10290_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel_name, wilson_steps):
    """Bytes per launch scaled from the small-case capture, or None when the
    kernel's sources changed since (or no capture exists for it)."""
    t = TRAFFIC_PER_WILSON_STEP.get(kernel_name.split()[0])
    if t is None or sources_sha1(t[1]) != t[2]:
        return None
    return t[0] * float(wilson_steps)


HEADLINE_METRIC = ("time to rel.err 1e-2 for all-node ECC+Kemeny; walk steps/s; CV vs plain, 1 GB300")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ba_1m", choices=["ba_1m", "er_1000", "rmat_22", "ba_200k", "ba_100k"])
    ap.add_argument("--batch", type=int, default=65536, help="samples per step")
    ap.add_argument("--seed", type=int, default=20231117)
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle baseline")
    ap.add_argument("--no-tta", action="store_true", help="skip the time-to-accuracy run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--ws-frac", type=float, default=0.6, help="fraction of free HBM lent as Wilson state")
    ap.add_argument("--ws-gb", type=float, default=0.0, help="cap on the Wilson-state workspace in GB (profiler runs)")
    ap.add_argument("--tta-large", default="ba_1m:16384:plain+paths+cv+cvpaths,rmat_22:65536:plain+cvpaths",
                    help="time to accuracy on large graphs: workload:largest omega of the grid[:forms joined by +], "
                         "comma separated (forms default to --tta-forms)")
    ap.add_argument("--tta-forms", default="plain,paths,cv",
                    help="estimator forms of the large-graph runs (plain, paths, cv, cvpaths: the control variate "
                         "with the loop-included paths)")
    ap.add_argument("--tta-seeds", type=int, default=10, help="seeds (disjoint id ranges) per form")
    ap.add_argument("--kernel", type=int, default=0, help="LAP_OPT_KERNEL for the timed steps (0: the library's choice)")
    ap.add_argument("--walkers", type=int, default=8, help="LAP_OPT_WALKERS (kernel 3)")
    ap.add_argument("--cv-graphs", type=int, default=200, help="training graphs for the learned control variate (0: skip)")
    ap.add_argument("--cv-batch", type=int, default=8192, help="samples per batch in the CV-vs-plain measurement")
    ap.add_argument("--batched-graphs", type=int, default=512, help="graphs of the uneven batch (0: skip)")
    ap.add_argument("--batched-samples", type=int, default=4096, help="samples per graph of the uneven batch")
    ap.add_argument("--batched-nmax", type=int, default=1_000_000, help="largest n of the uneven batch recipe")
    ap.add_argument("--batched-ws-gb", type=float, default=0.0, help="cap on the batch workspace in GB (profiler runs)")
    ap.add_argument("--batched-orders", default="0",
                    help="unit orders to time on the uneven batch: 0 largest first, 1 smallest first")
    ap.add_argument("--landmark-roots", type=int, default=6,
                    help="highest-degree roots of the landmark study on the BA 1e6 graph (0: skip)")
    ap.add_argument("--landmark-random", type=int, default=0,
                    help="random roots added to the landmark study (their absorbed walks to low-degree roots "
                         "run ~1e7 steps one after another: about 80 s for 256 samples)")
    ap.add_argument("--kemeny-sweep", type=int, default=1, help="kappa/n of 1e6-node BA and ER graphs (0: skip)")
    ap.add_argument("--study-samples", type=int, default=256, help="samples per root / graph of the two studies")
    ap.add_argument("--paths", type=int, default=1,
                    help="measure the loop-included-path form (LAP_OPT_PATHS) against own draws (0: skip)")
    ap.add_argument("--spantree-trees", type=int, default=4096,
                    help="SpanTree (Alg. 1/3) trees timed on the main workload (0: skip the SpanTree section)")
    ap.add_argument("--extra-workloads", default="rmat_22",
                    help="comma-separated extra single-graph workloads (plain throughput, CV vs plain)")
    ap.add_argument("--extra-samples", type=int, default=16384, help="samples per step of the extra workloads")
    ap.add_argument("--ceiling-probe", type=int, default=1,
                    help="measure the random 1-byte read+write ceiling the sampler is compared with (0: skip)")
    ap.add_argument("--extra-cv", type=int, default=0,
                    help="also measure the control variate against plain on the extra workloads (1: on)")
    return ap.parse_args()


KERNEL_NAMES = {1: "lewalk_kernel (8-byte state)", 2: "lewalk_compact_kernel (1-byte state)",
                3: "lewalk_group_kernel (several walkers per sample, 2-byte state)"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def load_graph(name):
    from paper_2311_10290_gb300 import inputs
    if name in ("ba_200k", "ba_100k"):   # smaller cases of the same family, for profiler captures
        g = inputs.ba(200_000 if name == "ba_200k" else 100_000, 5, seed=0)
        g.name = "ba_n%s_m5" % ("2e5" if name == "ba_200k" else "1e5")
        return g
    return {"ba_1m": inputs.ba_1m, "er_1000": inputs.er_1000, "rmat_22": inputs.rmat_22}[name]()


# ------------------------------------------------------------ clocks

class Clocks:
    """Samples nvidia-smi every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


# ------------------------------------------------------------ CPU oracle

def cpu_oracle_rate(g, v, seed, target_seconds, first_id=1 << 30):
    """The oracle as it stands, on all host cores (disjoint sample-id ranges),
    on a bounded number of samples of the same workload."""
    import oracle
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    c = oracle.sample(g.row_ptr, g.col, v, seed, first_id, 1, keep_per_sample=True)
    t1 = time.perf_counter() - t0
    per_sample = max(t1, 1e-4)
    per_core = max(1, int(target_seconds / per_sample))
    count = per_core * cores
    t0 = time.perf_counter()
    c = oracle.sample_threads(g.row_ptr, g.col, v, seed, first_id + 1, count, cores)
    dt = time.perf_counter() - t0
    steps = c.sum_y1 + int(c.cnt2.sum()) + c.sum_y2
    out = {"value": steps / dt, "unit": "walk steps/s", "cores": cores, "kind": "oracle",
           "sample": "%d samples (ids %d..%d) of the same graph and root, %d threads, %.1f s" %
                     (count, first_id + 1, first_id + count, cores, dt)}
    # One thread on a quarter of the per-core share, for the per-core rate.
    one = max(1, per_core // 4)
    t0 = time.perf_counter()
    c = oracle.sample(g.row_ptr, g.col, v, seed, first_id + 1 + count, one, keep_per_sample=False)
    dt1 = time.perf_counter() - t0
    steps1 = c.sum_y1 + int(c.cnt2.sum()) + c.sum_y2
    out["single_thread"] = {"value": steps1 / dt1, "unit": "walk steps/s",
                            "sample": "%d samples, 1 thread, %.1f s" % (one, dt1)}
    return out


def cpu_time_to_accuracy(omega, seed=7):
    """The oracle on all host cores at the omega the GPU's time-to-accuracy run
    found (same ids 0..omega-1 and seed as the GPU's timed run, so the same
    counts): wall seconds for sampling plus finalize, and the errors."""
    import oracle
    from paper_2311_10290_gb300 import inputs
    g = inputs.er_1000()
    ecc_t, kc_t, _ = read_truth()
    v = oracle.root_max_degree(g.row_ptr)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    c = oracle.sample_threads(g.row_ptr, g.col, v, seed, 0, omega, cores)
    _, ec, kc = oracle.finalize(g.row_ptr, v, omega, c.cnt1, c.cnt2, c.sum_y1, c.sum_y2)
    dt = time.perf_counter() - t0
    return {"omega": omega, "seconds": dt, "cores": cores, "kind": "oracle",
            "ecc_max_rel_err": float(np.max(np.abs(ec - ecc_t) / ecc_t)), "kc_rel_err": abs(kc - kc_t) / kc_t}


def cpu_oracle_extrapolated(g, v, seed, omega, sample=256, first_id=1 << 29):
    """The oracle on all host cores for a bounded sample of `sample` ids,
    extrapolated linearly to omega samples (the samples are independent and
    identically distributed, so the time grows in proportion)."""
    import oracle
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.sample_threads(g.row_ptr, g.col, v, seed, first_id, sample, cores)
    dt = time.perf_counter() - t0
    return {"omega": int(omega), "sample": sample, "sample_seconds": round(dt, 2), "cores": cores, "kind": "oracle",
            "seconds_extrapolated": dt * omega / sample,
            "note": "measured on %d sample ids, extrapolated linearly to omega" % sample}


# ------------------------------------------------------------ accuracy

def read_truth():
    path = os.path.join(ROOT, "tests", "golden", "dense_truth_er1000.txt")
    ecc, kc, meta = [], None, {}
    with open(path) as f:
        for line in f:
            if line.startswith("#"):
                continue
            k, val = line.split()
            if k == "ecc":
                ecc.append(float(val))
            elif k == "kemeny":
                kc = float(val)
            else:
                meta[k] = val
    return np.array(ecc), kc, meta


def time_to_accuracy(torch, LapGraph, seeds=10, target=1e-2, params=None, paths=0):
    """Smallest omega on the grid round(256 * 2^(k/4)) at which the mean over
    seeds of the ECC max relative error and of the Kemeny relative error are
    both <= 1e-2, on Erdos-Renyi G(1000, 0.01) against its dense FP64 truth;
    then the GPU time of one fresh run to that omega.  With `params` the
    estimates are the control-variate ones (potentials from the network,
    coefficients from pilot samples with disjoint ids)."""
    import hashlib
    from paper_2311_10290_gb300 import inputs
    g = inputs.er_1000()
    ecc_t, kc_t, meta = read_truth()
    h = hashlib.sha1()
    h.update(g.row_ptr.astype("<i4").tobytes())
    h.update(g.col.astype("<i4").tobytes())
    if h.hexdigest() != meta.get("sha1"):
        return {"error": "dense truth file does not match the generated graph"}
    pilot = 4096
    from paper_2311_10290_gb300.lap import LAP_OPT_PATHS
    handles = [LapGraph(g.row_ptr, g.col, workspace_bytes=8 * g.n * 65536) for _ in range(seeds)]
    betas = []
    for s, H in enumerate(handles):
        H.set_option(LAP_OPT_PATHS, paths)
        H.set_root()
        if params is not None:
            betas.append(cv_prepare(H, params, 500 + s, pilot=pilot, batches=4)[2:])

    def estimates(k, H):
        if params is None:
            return H.ecc(), H.kemeny()
        _, ec, kc, _ = H.cv_estimates(*betas[k])
        return ec, kc

    done, curve, found = 0, [], None
    for k in range(0, 53):
        target_omega = int(round(256 * 2.0 ** (k / 4.0)))
        e1, e2 = [], []
        for s, H in enumerate(handles):
            H.sample(target_omega - done, 1000 + s)
        for s, H in enumerate(handles):
            ec, kc = estimates(s, H)
            e1.append(float(np.max(np.abs(ec - ecc_t) / ecc_t)))
            e2.append(abs(kc - kc_t) / kc_t)
        done = target_omega
        curve.append((target_omega, float(np.mean(e1)), float(np.mean(e2))))
        if np.mean(e1) <= target and np.mean(e2) <= target:
            found = target_omega
            break
    for H in handles:
        H.close()
    label = "er_1000 (Erdos-Renyi G(1000,0.01), dense FP64 truth)"
    if found is None:
        return {"workload": label, "reached": False, "curve": curve}
    # The timed run gets the library's default workspace: on a 1000-node graph
    # that is more slots than samples, so every sample has its own lane and the
    # run lasts as long as its longest sample.
    H = LapGraph(g.row_ptr, g.col)
    H.set_option(LAP_OPT_PATHS, paths)
    H.set_root()
    prep = 0.0
    if params is not None:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b1, b2 = cv_prepare(H, params, 7777, pilot=pilot, batches=4)[2:]
        torch.cuda.synchronize()
        prep = time.perf_counter() - t0
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    H.sample(found, 7)
    if params is None:
        out = torch.empty(g.n, dtype=torch.float64, device="cuda")
        H.ecc(out)
        H.kemeny()
    else:
        H.cv_estimates(b1, b2)
    b.record()
    torch.cuda.synchronize()
    H.close()
    res = {"workload": label, "seeds": seeds, "omega": found, "gpu_seconds": a.elapsed_time(b) / 1e3,
           "ecc_max_rel_err_mean": curve[-1][1], "kc_rel_err_mean": curve[-1][2],
           "curve": [{"omega": o, "ecc_max_rel": round(x, 5), "kc_rel": round(y, 6)} for o, x, y in curve]}
    if params is not None:
        res["pilot_samples"] = pilot + min(pilot, 4096)
        res["prepare_seconds"] = round(prep, 3)
        res["note"] = ("gpu_seconds: CV sampling + CV finalize at omega; prepare_seconds: pilot samples, "
                       "features, MLP forward and coefficient fit (wall)")
    return res


# First sample id of each estimator form in the large-graph time-to-accuracy
# runs: seed s of a form takes [base + s * omega_max, base + (s + 1) * omega_max),
# its timed call [base + TTA_TIMED_OFFSET, ... + omega); all disjoint below 2^32.
TTA_ID_BASE = {"plain": 0, "paths": 1 << 30, "cv": (1 << 30) + (1 << 29), "cvpaths": 1 << 31}
TTA_TIMED_OFFSET = 1 << 28


def omega_grid(omega_max, lo=256):
    """round(lo * 2^(k/2)) up to omega_max (the last point is omega_max)."""
    out, k = [], 0
    while True:
        w = int(round(lo * 2.0 ** (k / 2.0)))
        if w >= omega_max:
            out.append(int(omega_max))
            return out
        out.append(w)
        k += 1


class CheckpointBlocks:
    """One handle per block of the omega grid, each on its own CUDA stream, so
    that every block of a seed samples at once: the estimate at grid point k
    is the sum of blocks 0..k, i.e. the sample ids [first, first + grid[k]).
    A further handle (which never samples) finalizes the running sums with
    the library (lap_set_counts, lap_cv_set_sums, lap_ecc / lap_cv_estimates)."""

    def __init__(self, torch, LapGraph, g, v, grid, form, ws_total, phi=None):
        from paper_2311_10290_gb300.lap import LAP_OPT_PATHS
        self.torch, self.g, self.v, self.grid, self.form, self.phi = torch, g, v, grid, form, phi
        self.bounds = [0] + list(grid)
        sizes = [self.bounds[k + 1] - self.bounds[k] for k in range(len(grid))]
        self.streams = [torch.cuda.Stream() for _ in sizes]
        self.handles = []
        # Lanes are shared out in proportion to the block sizes, so that the
        # blocks' kernels fit on the GPU together and run side by side.
        from paper_2311_10290_gb300.lap import LAP_OPT_SLOTS, LAP_OPT_WALKERS
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        lanes = sms * 1024
        paths = form in ("paths", "cvpaths")
        walkers = 8                                    # kernel 3 counts groups of 8 lanes as one slot
        for k, sz in enumerate(sizes):
            ws = max(8 * g.n * 4, int(ws_total * sz / grid[-1]))
            H = LapGraph(g.row_ptr, g.col, workspace_bytes=ws, stream=self.streams[k])
            H.set_option(LAP_OPT_PATHS, 1 if paths else 0)
            H.set_option(LAP_OPT_WALKERS, 8)
            H.set_option(LAP_OPT_SLOTS, max(1, int(lanes / walkers * sz / grid[-1])))
            self.handles.append(H)
        self.F = LapGraph(g.row_ptr, g.col, workspace_bytes=8 * g.n)
        self.F.set_root(v)
        if phi is not None:
            self.F.cv_set_potentials(*phi)

    def close(self):
        for H in self.handles + [self.F]:
            H.close()

    def run(self, first, seed, betas=None):
        """All blocks of one seed; returns (list of (ECC tensor float32 on the
        device, Kemeny) per grid point, final (cnt1 int64, sum Y1))."""
        from paper_2311_10290_gb300.lap import LAP_OPT_CURSOR
        torch, g = self.torch, self.g
        for k, H in enumerate(self.handles):
            H.set_root(self.v)
            H.set_option(LAP_OPT_CURSOR, first + self.bounds[k])
            if self.phi is not None:
                H.cv_set_potentials(*self.phi)
            H.sample(self.bounds[k + 1] - self.bounds[k], seed)
        c1 = np.zeros(g.n, dtype=np.uint64)
        c2 = np.zeros(g.n, dtype=np.uint64)
        sums = np.zeros(3, dtype=np.uint64)
        a = [np.zeros(g.n, dtype=np.int64) for _ in range(3)] if self.phi is not None else None
        est = torch.empty(g.n, dtype=torch.float64, device="cuda")
        out = []
        for k, H in enumerate(self.handles):
            b1, b2, bs = H.counts()
            c1 += b1
            c2 += b2
            sums += bs[:3]
            self.F.set_counts(c1, c2, sums)
            if a is None:
                self.F.ecc(est)
                kc = self.F.kemeny()
            else:
                for x, y in zip(a, H.cv_sums()):
                    x += y
                self.F.cv_set_sums(*a)
                _, _, kc, _ = self.F.cv_estimates(*betas, ecc_out=est)
            out.append((est.float().clone(), kc))
        return out, (c1.astype(np.int64), int(sums[1]))


def exact_parts(torch, LapGraph, g, v, rtol=1e-12):
    """The parts of the large-graph ground truth that one FP64 solve each
    fixes, by the library's conjugate-gradient solver (lap_lv_solve):
    y2(u) = (L_v^{-1} 1)_u / n, lvv = (L^+)_vv = (1/n) sum_u y2(u), and
    E[Y2] = d^T L_v^{-1} d / 2m."""
    H = LapGraph(g.row_ptr, g.col, workspace_bytes=8 * g.n)
    try:
        H.set_root(v)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d = torch.from_numpy(np.diff(g.row_ptr.astype(np.int64)).astype(np.float64)).cuda()
        r1, it1, res1 = H.lv_solve(torch.ones(g.n, dtype=torch.float64, device="cuda"), rtol=rtol)
        hv, it2, res2 = H.lv_solve(d, rtol=rtol)
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
    finally:
        H.close()
    y2 = r1 / g.n
    return {"y2": y2, "lvv": float(y2.sum().item()) / g.n, "ey2": float((d * hv).sum().item()) / float(g.arcs),
            "info": {"iterations": [it1, it2], "residuals": [res1, res2], "seconds": round(secs, 3), "rtol": rtol}}


def ecc_truth(torch, g, v, cnt1, omega_pool, sum_y1, exact):
    """ECC and Kemeny ground truth from pooled plain counts plus the exact
    parts of the sparse solves: (L^+)_uu = cnt1_pool(u) / (omega_pool d_u)
    - 2 y2(u) + lvv (u != v), (L^+)_vv = lvv (Section 3.1, element-wise
    Theorem 1), c(u) = (n-1) / (n (L^+)_uu + Tr L^+) (Section 2), and
    kappa = sum Y1 / omega_pool - E[Y2] (Alg. 4)."""
    d = torch.from_numpy(np.diff(g.row_ptr.astype(np.int64)).astype(np.float64)).cuda()
    ld = torch.from_numpy(cnt1).cuda().double() / (float(omega_pool) * d) - 2.0 * exact["y2"] + exact["lvv"]
    ld[v] = exact["lvv"]
    ecc = (g.n - 1) / (g.n * ld + ld.sum())
    kc = float(sum_y1) / float(omega_pool) - exact["ey2"]
    return ecc.float(), kc


def timed_run(torch, LapGraph, g, v, omega, first, seed, form, phi=None, betas=None):
    """One fresh call of omega samples (the library's kernel choice) plus the
    finalize, timed with CUDA events on the handle's stream; with its
    algorithmic bytes and roofline fraction."""
    from paper_2311_10290_gb300.lap import LAP_OPT_CURSOR, LAP_OPT_PATHS, LAP_STAT_LAST_KERNEL
    H = LapGraph(g.row_ptr, g.col, workspace_bytes=int(torch.cuda.mem_get_info()[0] * 0.5))
    try:
        H.set_option(LAP_OPT_PATHS, 1 if form in ("paths", "cvpaths") else 0)
        H.set_root(v)
        H.set_option(LAP_OPT_CURSOR, first)
        if phi is not None:
            H.cv_set_potentials(*phi)
        est = torch.empty(g.n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        H.sample(omega, seed)
        if phi is None:
            H.ecc(est)
            H.kemeny()
        else:
            H.cv_estimates(*betas, ecc_out=est)
        b.record()
        torch.cuda.synchronize()
        secs = a.elapsed_time(b) / 1e3
        _, c2, sums = H.counts()
        kernel = H.stat(LAP_STAT_LAST_KERNEL)
    finally:
        H.close()
    alg = (BYTES_WILSON_STEP * int(sums[1]) + BYTES_TREE_INSERT * (g.n - 1) * omega +
           BYTES_WALK_STEP * (int(c2.sum()) + int(sums[2])))
    pk = peaks()[0]
    return {"gpu_seconds": secs, "kernel": kernel, "walk_steps": int(sums[1]) + int(c2.sum()) + int(sums[2]),
            "roofline": {"bound": "hbm", "achieved": alg / secs / 1e9, "peak": pk, "unit": "GB/s",
                         "frac": alg / secs / 1e9 / pk,
                         "note": "algorithmic bytes of the timed call (sampling plus finalize) over its time"}}


def time_to_accuracy_large(torch, LapGraph, g, v, exact, omega_max, forms=("plain", "paths", "cv"), params=None,
                           seeds=10, target=1e-2, ws_frac=0.5):
    """Time to relative error 1e-2 on a large graph, Section 6's protocol:
    ECC max relative error over all nodes and Kemeny relative error, each the
    mean over `seeds` seeds (disjoint sample-id ranges), on the grid
    round(256 * 2^(k/2)) up to omega_max; the smallest grid point where both
    means are <= target, then one fresh timed call to it.

    Ground truth: the plain estimates pooled over the plain seeds (all of
    them for the other forms, whose ids are disjoint; all but the seed itself
    for a plain seed), with the parts the sparse solves fix exactly (y2,
    L^+_vv, E[Y2]).  The pool holds at least (seeds - 1) * omega_max samples."""
    res = {"seeds": seeds, "grid_max": omega_max, "target": target}
    grid = omega_grid(omega_max)
    ws_total = int(torch.cuda.mem_get_info()[0] * ws_frac)
    stored, finals = [], []
    base = TTA_ID_BASE
    for form in forms:
        if form in ("cv", "cvpaths") and params is None:
            continue
        t0 = time.perf_counter()
        phi = betas = None
        prep = 0.0
        if form in ("cv", "cvpaths"):
            from paper_2311_10290_gb300.lap import LAP_OPT_PATHS
            from paper_2311_10290_gb300.lap import LapGraph as LG
            P = LG(g.row_ptr, g.col, workspace_bytes=int(torch.cuda.mem_get_info()[0] * 0.3))
            try:
                # The coefficients are fitted on pilot samples of the same form.
                P.set_option(LAP_OPT_PATHS, 1 if form == "cvpaths" else 0)
                P.set_root(v)
                torch.cuda.synchronize()
                tp = time.perf_counter()
                phi1, phi2, b1, b2 = cv_prepare(P, params, 4242, pilot=8192, batches=8)
                torch.cuda.synchronize()
                prep = time.perf_counter() - tp
            finally:
                P.close()
            phi, betas = (phi1, phi2), (b1, b2)
        blocks = CheckpointBlocks(torch, LapGraph, g, v, grid, form, ws_total, phi=phi)
        per_seed = []
        try:
            for s in range(seeds):
                curve, fin = blocks.run(base[form] + s * omega_max, 1, betas)
                per_seed.append(curve)
                if form == "plain":
                    finals.append(fin)
        finally:
            blocks.close()
        stored.append((form, per_seed, phi, betas, prep, time.perf_counter() - t0))
    if not finals:
        return {"error": "the plain form is needed for the ground truth"}
    pool_c = sum(c for c, _ in finals)
    pool_y = sum(y for _, y in finals)
    for form, per_seed, phi, betas, prep, wall in stored:
        errs = np.zeros((seeds, len(grid), 2))
        for s, curve in enumerate(per_seed):
            if form == "plain":
                c, y = pool_c - finals[s][0], pool_y - finals[s][1]
                ecc_t, kc_t = ecc_truth(torch, g, v, c, (seeds - 1) * omega_max, y, exact)
            elif s == 0:
                ecc_t, kc_t = ecc_truth(torch, g, v, pool_c, seeds * omega_max, pool_y, exact)
            for j, (est, kc) in enumerate(curve):
                errs[s, j, 0] = float(torch.max(torch.abs(est - ecc_t) / ecc_t))
                errs[s, j, 1] = abs(kc - kc_t) / abs(kc_t)
        mean = errs.mean(axis=0)
        found = next((w for j, w in enumerate(grid) if mean[j, 0] <= target and mean[j, 1] <= target), None)
        r = {"curve": [{"omega": w, "ecc_max_rel": round(float(mean[j, 0]), 5), "kc_rel": round(float(mean[j, 1]), 7)}
                       for j, w in enumerate(grid)],
             "truth_samples": (seeds - 1 if form == "plain" else seeds) * omega_max, "wall_seconds": round(wall, 1)}
        if form in ("cv", "cvpaths"):
            r["betas"] = list(betas)
            r["prepare_seconds"] = round(prep, 2)
        if found is None:
            # Beyond the grid: the errors fall like omega^(-1/2); the fit over
            # the last four grid points gives the omega the target needs.
            ws = np.array(grid[-4:], dtype=np.float64)
            e = np.maximum(mean[-4:, 0], mean[-4:, 1])
            c = float(np.exp(np.mean(np.log(e) + 0.5 * np.log(ws))))
            r.update({"reached": False, "omega_extrapolated": int(math.ceil((c / target) ** 2)),
                      "note": "not reached on the grid; omega_extrapolated = (c / target)^2 from err = c / sqrt(omega) "
                              "fitted to the last four grid points"})
        else:
            j = grid.index(found)
            r.update({"reached": True, "omega": found, "ecc_max_rel_err_mean": float(mean[j, 0]),
                      "kc_rel_err_mean": float(mean[j, 1])})
            r.update(timed_run(torch, LapGraph, g, v, found, base[form] + TTA_TIMED_OFFSET, 1, form, phi=phi,
                               betas=betas))
        res[form] = r
    return res


def note(msg):
    """Progress line on stderr (the JSON result goes alone to stdout)."""
    print("[bench %.1fs] %s" % (time.perf_counter() - _T0, msg), file=sys.stderr, flush=True)


_T0 = time.perf_counter()


# ------------------------------------------------------------ learned CV

def cv_training_set(count, seed0=1000):
    """Training graphs: Barabasi-Albert (m in 3..10) and R-MAT, n log-uniform in [1e4, 1e5]."""
    from paper_2311_10290_gb300 import inputs
    out = []
    for k in range(count):
        s = seed0 + k
        h = np.random.Generator(np.random.PCG64(s))
        n = int(round(math.exp(h.uniform(math.log(1e4), math.log(1e5)))))
        if k % 2 == 0:
            out.append(inputs.ba(n, 3 + (k // 2) % 8, seed=s))
        else:
            out.append(inputs.rmat(max(10, int(math.ceil(math.log2(n)))), 8, seed=s))
    return out


def cv_train(torch, LapGraph, count):
    """Targets from the sampler on `count` generated graphs, then AdamW training
    of the MLP on the library's BF16 tensor-core kernels."""
    from paper_2311_10290_gb300 import cv as CVG
    t0 = time.perf_counter()
    sets, rows = [], 0
    for tg in cv_training_set(count):
        G = LapGraph(tg.row_ptr, tg.col, workspace_bytes=int(4e9))
        G.set_root()
        sets.append(CVG.training_targets(G, omega=512, reps=16, seed=11))
        rows += tg.n - 1
        G.close()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    params, hist = CVG.train(sets, epochs=8, batch=8192)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return params, {"training_graphs": count, "training_rows": rows,
                    "training": "BA (m 3..10) and R-MAT (edge factor 8), n log-uniform in [1e4, 1e5], seeds from 1000; "
                                "targets from the sampler: 512 Wilson samples and 16 v-absorbed walks per node",
                    "data_seconds": round(t1 - t0, 2), "train_seconds": round(t2 - t1, 2),
                    "loss_first_last_epoch": [round(hist[0], 5), round(hist[-1], 5)]}


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


# Useful (unpadded) products per row of the 8 -> 64 -> 64 -> 2 network:
# forward 2 (8*64 + 64*64 + 64*2); the backward adds dY W3, dH2 W2 and the
# three weight gradients.
MLP_FLOP_FWD = 2 * (8 * 64 + 64 * 64 + 64 * 2)
MLP_FLOP_TRAIN = MLP_FLOP_FWD + 2 * (2 * 64 + 64 * 64 + 64 * 64 + 64 * 8 + 2 * 64)


def mlp_kernel_timing(torch, rows_list=(8192, 1 << 22), reps=20):
    """CUDA-event time of the MLP kernels on random rows: the tcgen05 kernel
    (TMEM accumulators) beside the mma.sync kernel, forward and loss+gradient,
    with the useful tensor FLOP/s and the HBM bytes (X and Y or T) per second
    against the measured peaks."""
    from paper_2311_10290_gb300 import lap as L
    hbm, hbm_kind = peaks()
    tc, tc_kind = bf16_peak()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    P = torch.randn(L.LAP_MLP_PARAMS, device="cuda", generator=gen) * 0.1
    st = torch.cuda.current_stream()
    rows_out = []
    try:
        for rows in rows_list:
            X = torch.randn(rows, 8, device="cuda", generator=gen)
            T = torch.randn(rows, 2, device="cuda", generator=gen)
            Y = torch.empty(rows, 2, device="cuda")
            G = torch.zeros(L.LAP_MLP_PARAMS, device="cuda")
            loss = torch.zeros(1, device="cuda")
            for kname, k in (("tcgen05", L.LAP_MLP_TCGEN05), ("mma_sync", L.LAP_MLP_MMA_SYNC)):
                L.lap_mlp_select(k)
                calls = (("forward", MLP_FLOP_FWD, lambda: L.lap_mlp_forward(P, X, rows, Y, st.cuda_stream)),
                         ("loss_grad", MLP_FLOP_TRAIN,
                          lambda: L.lap_mlp_loss_grad(P, X, T, rows, 1.0, 1.0, G, loss, st.cuda_stream)))
                for what, flop, fn in calls:
                    for _ in range(3):
                        fn()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(st)
                    for _ in range(reps):
                        fn()
                    e1.record(st)
                    e1.synchronize()
                    ms = e0.elapsed_time(e1) / reps
                    tflops = flop * rows / (ms * 1e-3) / 1e12
                    gbs = 40.0 * rows / (ms * 1e-3) / 1e9
                    rows_out.append({"kernel": kname, "call": what, "rows": rows, "ms": round(ms, 4),
                                     "rows_per_s": rows / (ms * 1e-3), "tflops": round(tflops, 2),
                                     "tensor_frac": round(tflops / tc, 4), "hbm_gbs": round(gbs, 1),
                                     "hbm_frac": round(gbs / hbm, 4)})
            del X, T, Y, G, loss
    finally:
        L.lap_mlp_select(L.LAP_MLP_TCGEN05)
    return {"rows": rows_out, "flop_per_row": {"forward": MLP_FLOP_FWD, "loss_grad": MLP_FLOP_TRAIN},
            "bytes_per_row": 40, "peaks": {"bf16_tflops": tc, "bf16_kind": tc_kind, "hbm_gbs": hbm,
                                           "hbm_kind": hbm_kind},
            "note": "each call is one launch; forward reads X (32 B) and writes Y (8 B) per row, loss+gradient "
                    "reads X and T; 8192 rows is the training batch"}


def cv_diagnostics(torch, LapGraph, params, graphs=None, omega=1 << 18, samples=8192):
    """What the trained network learned, on held-out graphs small enough for
    near-exact targets: R^2 of head 0 against the mean Wilson visits of
    `omega` samples (d_u (L_v^{-1})_uu, standard error about 1e-3), R^2 of
    head 1 against the exact h(u, v) / E[Y2] of the library's FP64 solve; and
    the per-sample variance of the Kemeny estimator Y1 - Y2 + beta2 M2
    relative to plain with (a) the network's potential, (b) the exact
    hitting-time potential (the best any potential can do for the pi-walk
    term: Y2 - M2 is then the start's hitting time), each also on the
    loop-included paths."""
    from paper_2311_10290_gb300 import cv as CVG
    from paper_2311_10290_gb300 import inputs
    from paper_2311_10290_gb300.lap import LAP_OPT_CURSOR, LAP_OPT_PATHS
    graphs = graphs or [inputs.ba(3000, 4, seed=9001), inputs.rmat(11, 8, seed=9002)]
    out = []
    for g in graphs:
        G = LapGraph(g.row_ptr, g.col, workspace_bytes=1 << 30)
        try:
            v = G.set_root()
            d = torch.from_numpy(np.diff(g.row_ptr.astype(np.int64)).astype(np.float64)).cuda()
            G.sample(omega, 1)
            c1, _, sums = G.counts()
            ey2 = float(sums[2]) / omega
            hv, _, _ = G.lv_solve(d)
            ey2_exact = float((d * hv).sum().item()) / float(g.arcs)
            y = CVG.predict(G, params).double()
            keep = torch.ones(g.n, dtype=torch.bool, device="cuda")
            keep[v] = False
            t0 = torch.from_numpy(c1.astype(np.float64) / omega).cuda()
            t1 = hv / ey2_exact

            def r2(pred, t):
                return float(1.0 - ((pred - t) ** 2).sum() / ((t - t.mean()) ** 2).sum())

            row = {"graph": g.name, "n": g.n, "r2_visits_head": r2(y[keep, 0], t0[keep]),
                   "r2_hitting_head": r2(y[keep, 1], t1[keep]), "mean_y2_sampled": ey2, "mean_y2_exact": ey2_exact}
            exact_phi2 = hv.clone()
            exact_phi2[v] = 0.0
            for paths in (0, 1):
                for name, phi2 in (("network", None), ("exact_hitting_time", exact_phi2)):
                    G.set_root(v)
                    G.set_option(LAP_OPT_PATHS, paths)
                    if phi2 is None:
                        p1, p2 = CVG.pilot_potentials(G, params, seed=3, samples=2048)
                    else:
                        p1, p2 = None, phi2
                    _, b2 = CVG.fit_betas(G, p1, p2, seed=4, pilot=8192)
                    G.set_root(v)
                    G.set_option(LAP_OPT_CURSOR, 1 << 24)
                    G.cv_set_potentials(p1, p2)
                    a, b, m = G.sample_trace_cv(samples, 5)
                    est = (a - b).double()
                    cvv = est + b2 * m
                    row["kemeny_var_ratio_%s%s" % (name, "_paths" if paths else "")] = float(cvv.var() / est.var())
                    row["kemeny_var_plain%s" % ("_paths" if paths else "")] = float(est.var())
        finally:
            G.close()
        out.append(row)
    return out


def cv_prepare(G, params, seed, pilot, batches):
    """Potentials from the network, coefficients from pilot samples (disjoint ids)."""
    from paper_2311_10290_gb300 import cv as CVG
    phi1, phi2 = CVG.pilot_potentials(G, params, seed + 1, samples=min(pilot, 4096))
    beta1, beta2 = CVG.fit_betas(G, phi1, phi2, seed=seed, pilot=pilot, batches=batches)
    return phi1, phi2, beta1, beta2


def _neighbour_sums_of_potential(g, phi1):
    """Measurement helper: S1(u) = sum over N(u) of round(2^16 phi1), the
    neighbour sums the library forms for its Wilson-draw variate, to split the
    per-batch visit counts into their control-variate parts."""
    h = np.rint(np.ldexp(phi1.cpu().numpy(), 16)).astype(np.int64)
    rp = g.row_ptr.astype(np.int64)
    src = np.repeat(np.arange(g.n), rp[1:] - rp[:-1])
    out = np.zeros(g.n, dtype=np.int64)
    np.add.at(out, src, h[g.col])
    return out.astype(np.float64)


def cv_measurement(torch, LapGraph, g, v, params, samples_per_batch, batches):
    """Samples needed for the same variance, CV against plain, on one graph:
    Kemeny from per-sample traces; ECC from per-node variances of the visit
    estimator between `batches` independent batches.  The coefficients come
    from separate pilot samples, so both estimators stay unbiased."""
    from paper_2311_10290_gb300.lap import LAP_OPT_CURSOR, lap_counts
    free, _ = torch.cuda.mem_get_info()
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=int(free * 0.5))
    try:
        G.set_root(v)                             # plain and CV: the library's kernel choice for the same calls
        t0 = time.perf_counter()
        phi1, phi2, beta1, beta2 = cv_prepare(G, params, 4242, pilot=2 * samples_per_batch, batches=4)
        t_prep = time.perf_counter() - t0
        # Kemeny: per-sample Y1 - Y2 and M2 on fresh samples.
        a, b, m = G.sample_trace_cv(samples_per_batch, 31337)
        est = (a - b).double().cpu().numpy()
        cvv = est + beta2 * m.cpu().numpy()
        kc_ratio = float(np.var(cvv) / np.var(est))
        # ECC: per-node visit estimator in `batches` batches (fresh ids).
        G.set_root(v)
        G.set_option(LAP_OPT_CURSOR, samples_per_batch)          # ids after the Kemeny trace's
        d = np.diff(g.row_ptr.astype(np.int64)).astype(np.float64)
        s1 = _neighbour_sums_of_potential(g, phi1)
        prev_c, prev_a = np.zeros(g.n), np.zeros(g.n)
        V, Z = [], []
        for _ in range(batches):
            G.sample(samples_per_batch, 31337)
            c1, _, _ = lap_counts(G.h, g.n)
            a1, _, _ = G.cv_sums()
            c1, a1 = c1.astype(np.float64), a1.astype(np.float64)
            dc, da = c1 - prev_c, a1 - prev_a
            prev_c, prev_a = c1, a1
            V.append(dc)
            Z.append((d * da - dc * s1) / d)
        V, Z = np.array(V), np.array(Z)
        keep = np.ones(g.n, bool)
        keep[v] = False
        vp = V.var(axis=0, ddof=1)[keep]
        vc = (V - beta1 * Z).var(axis=0, ddof=1)[keep]
        ok = vp > 0
        per_node = vc[ok] / vp[ok]
        # Sampler cost with and without the CV terms (same ids, same graph).
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        G.set_root(v)
        ev[0].record()
        G.sample(samples_per_batch, 5)
        ev[1].record()
        G.set_root(v)
        G.cv_set_potentials(None, None)
        ev[2].record()
        G.sample(samples_per_batch, 5)
        ev[3].record()
        torch.cuda.synchronize()
        t_cv, t_plain = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    finally:
        G.close()
    return {"workload": g.name, "beta1": beta1, "beta2": beta2, "prepare_seconds": round(t_prep, 2),
            "pilot_samples": 2 * samples_per_batch + min(2 * samples_per_batch, 4096),
            "kemeny_samples_ratio": kc_ratio,
            "ecc_visit_samples_ratio_total": float(vc[ok].sum() / vp[ok].sum()),
            "ecc_visit_samples_ratio_median_node": float(np.median(per_node)),
            "cv_sampler_time_ratio": t_cv / t_plain,
            "kemeny_time_ratio_same_error": kc_ratio * t_cv / t_plain,
            "protocol": "%d fresh samples for Kemeny (per-sample variance); %d batches of %d for per-node "
                        "visit-count variance; ratios CV/plain on the same samples" % (samples_per_batch, batches,
                                                                                     samples_per_batch)}


# ------------------------------------------------------------ loop-included paths

def paths_measurement(torch, LapGraph, g, v, args, samples=8192, batches=4):
    """LAP_OPT_PATHS = 1 against own draws on one graph: per-sample variance
    of Y1 - Y2 (Kemeny), per-node variance of the L^+_uu numerator
    (cnt1 - 2 cnt2) / d between batches (ECC), and sampler time."""
    from paper_2311_10290_gb300.lap import LAP_OPT_CURSOR, LAP_OPT_PATHS, LAP_STAT_LAST_KERNEL, lap_counts
    free, _ = torch.cuda.mem_get_info()
    out = {"workload": g.name, "samples": samples, "batches": batches}
    d = np.diff(g.row_ptr.astype(np.int64)).astype(np.float64)
    keep = np.ones(g.n, bool)
    keep[v] = False
    res = {}
    for mode in (0, 1):
        G = LapGraph(g.row_ptr, g.col, workspace_bytes=int(free * 0.5))
        try:
            G.set_option(LAP_OPT_PATHS, mode)             # the library's kernel choice in both modes
            G.set_root(v)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            y1, y2 = G.sample_trace(samples, args.seed)
            b.record()
            torch.cuda.synchronize()
            t = a.elapsed_time(b) / 1e3
            out["kernel_paths%d" % mode] = G.stat(LAP_STAT_LAST_KERNEL)
            kvar = float(np.var((y1 - y2).double().cpu().numpy()))
            G.set_root(v)
            G.set_option(LAP_OPT_CURSOR, samples)
            prev1, prev2, rows = np.zeros(g.n), np.zeros(g.n), []
            for _ in range(batches):
                G.sample(samples, args.seed)
                c1, c2, _ = lap_counts(G.h, g.n)
                c1, c2 = c1.astype(np.float64), c2.astype(np.float64)
                rows.append(((c1 - prev1) - 2.0 * (c2 - prev2)) / d)
                prev1, prev2 = c1, c2
            ev = np.array(rows).var(axis=0, ddof=1)[keep]
        finally:
            G.close()
        res[mode] = (t, kvar, ev)
    t0, k0, e0 = res[0]
    t1, k1, e1 = res[1]
    ok = e0 > 0
    out.update({"kemeny_samples_ratio": k1 / k0, "ecc_numerator_samples_ratio_total": float(e1[ok].sum() / e0[ok].sum()),
                "ecc_numerator_samples_ratio_median_node": float(np.median(e1[ok] / e0[ok])),
                "sampler_time_ratio": t1 / t0, "sampler_seconds_own_draws": t0, "sampler_seconds_paths": t1,
                "kemeny_time_ratio_same_error": k1 / k0 * t1 / t0})
    return out


# ------------------------------------------------------------ SpanTree (Alg. 1, Alg. 3)

def spantree_tta(torch, LapGraph, seeds=10, target=1e-2):
    """Time-to-accuracy of the SpanTree estimators on Erdos-Renyi G(1000, 0.01)
    against the dense truth (same protocol and omega grid as the plain form)."""
    import hashlib
    from paper_2311_10290_gb300 import inputs
    g = inputs.er_1000()
    ecc_t, kc_t, meta = read_truth()
    h = hashlib.sha1()
    h.update(g.row_ptr.astype("<i4").tobytes())
    h.update(g.col.astype("<i4").tobytes())
    if h.hexdigest() != meta.get("sha1"):
        return {"error": "dense truth file does not match the generated graph"}
    handles = [LapGraph(g.row_ptr, g.col, workspace_bytes=8 * g.n * 32768) for _ in range(seeds)]
    for H in handles:
        H.set_root()
    done, curve, found = 0, [], None
    for k in range(0, 49):
        target_omega = int(round(256 * 2.0 ** (k / 4.0)))
        e1, e2 = [], []
        for sd, H in enumerate(handles):
            H.spantree_sample(target_omega - done, 1000 + sd)
        for H in handles:
            _, ec, kc = H.spantree_estimates()
            e1.append(float(np.max(np.abs(ec - ecc_t) / ecc_t)))
            e2.append(abs(kc - kc_t) / kc_t)
        done = target_omega
        curve.append((target_omega, float(np.mean(e1)), float(np.mean(e2))))
        if np.mean(e1) <= target and np.mean(e2) <= target:
            found = target_omega
            break
    for H in handles:
        H.close()
    label = "er_1000 (Erdos-Renyi G(1000,0.01), dense FP64 truth)"
    if found is None:
        return {"workload": label, "reached": False,
                "curve": [{"omega": o, "ecc_max_rel": round(x, 5), "kc_rel": round(y, 6)} for o, x, y in curve]}
    H = LapGraph(g.row_ptr, g.col, workspace_bytes=8 * g.n * 32768)
    H.set_root()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    H.spantree_sample(found, 7)
    H.spantree_estimates()
    b.record()
    torch.cuda.synchronize()
    H.close()
    return {"workload": label, "seeds": seeds, "omega": found, "gpu_seconds": a.elapsed_time(b) / 1e3,
            "ecc_max_rel_err_mean": curve[-1][1], "kc_rel_err_mean": curve[-1][2],
            "curve": [{"omega": o, "ecc_max_rel": round(x, 5), "kc_rel": round(y, 6)} for o, x, y in curve]}


def spantree_measurement(torch, LapGraph, g, v, args):
    """SpanTree throughput on the main workload (trees/s and per-tree cost
    against the LEWalk sampler's per-sample cost), then its time to accuracy
    on the small workload."""
    free, _ = torch.cuda.mem_get_info()
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=int(free * 0.5))
    try:
        G.set_root(v)
        G.spantree_sample(256, args.seed)             # warm-up (allocations, BFS parents)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        G.spantree_sample(args.spantree_trees, args.seed)
        b.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 1e3
        _, _, kc = G.spantree_estimates()
    finally:
        G.close()
    return {"workload": g.name, "trees": args.spantree_trees, "seconds": t, "trees_per_s": args.spantree_trees / t,
            "kemeny_estimate": kc, "time_to_accuracy": spantree_tta(torch, LapGraph),
            "note": "trees: 8-byte Wilson kernel, one tree per lane, then one CTA per tree for the flow sums "
                    "(children, levels, subtree sizes, preorder intervals, BFS-path sums)"}


# ------------------------------------------------------------ studies (batched runtime)

def landmark_study(torch, g, args):
    """Section 6 landmark study on one graph: Tr((I - P_v)^{-1}) (the expected
    cost of a Wilson run, estimated by sum Y1 / omega) and Kemeny's constant
    for the highest-degree roots and for random roots, all roots in one
    batched launch sharing one copy of the CSR."""
    from paper_2311_10290_gb300.lap import LapBatch
    deg = np.diff(g.row_ptr.astype(np.int64))
    n_rand = args.landmark_random
    top = [int(x) for x in np.argsort(-deg, kind="stable")[:max(1, args.landmark_roots)]]
    rng = np.random.Generator(np.random.PCG64(7))
    rand = [int(x) for x in rng.choice(g.n, size=n_rand, replace=False)]
    roots = top + rand
    t0 = time.perf_counter()
    B = LapBatch([(g.row_ptr, g.col)] * len(roots), roots=roots)
    try:
        B.autotune(args.study_samples, args.seed, window_ms=100.0)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        B.run(args.study_samples, args.seed)
        B.sync()
        b.record()
        torch.cuda.synchronize()
        tr = B.mean_wilson_steps() / g.n
        kc = B.kemeny()
    finally:
        B.close()
    rows = [{"root": v, "degree": int(deg[v]), "tr_over_n": round(float(t), 4), "kemeny": round(float(k), 1)}
            for v, t, k in zip(roots, tr, kc)]
    return {"graph": g.name, "roots": len(roots), "samples_per_root": args.study_samples,
            "gpu_seconds": a.elapsed_time(b) / 1e3, "wall_seconds": round(time.perf_counter() - t0, 2),
            "best_root": rows[int(np.argmin(tr))], "max_degree_root": rows[0],
            "tr_over_n_random_roots": {"min": float(np.min(tr[len(top):])) if rand else None,
                                       "median": float(np.median(tr[len(top):])) if rand else None,
                                       "max": float(np.max(tr[len(top):])) if rand else None},
            "rows": rows}


def kemeny_sweep(torch, args):
    """Kemeny's constant per node of 1e6-node Barabasi-Albert (m = 2, 3, 5, 8)
    and Erdos-Renyi (average degree 4, 8, 16, 32) graphs, one batched launch
    (the paper's synthetic-graph Kemeny experiment, Section 6)."""
    from paper_2311_10290_gb300 import inputs
    from paper_2311_10290_gb300.lap import LapBatch
    spec = [("ba", 1_000_000, 2.0 * m, 900 + m) for m in (2, 3, 5, 8)] + \
           [("er", 1_000_000, float(d), 950 + d) for d in (4, 8, 16, 32)]
    t0 = time.perf_counter()
    graphs = inputs.batch_graphs(spec)
    t_gen = time.perf_counter() - t0
    B = LapBatch([(x.row_ptr, x.col) for x in graphs])
    try:
        B.autotune(args.study_samples, args.seed, window_ms=100.0)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        B.run(args.study_samples, args.seed)
        B.sync()
        b.record()
        torch.cuda.synchronize()
        kc = B.kemeny()
        tr = B.mean_wilson_steps()
    finally:
        B.close()
    rows = [{"family": f, "avg_degree": d, "n": x.n, "arcs": x.arcs, "kemeny_over_n": round(float(k) / x.n, 4),
             "tr_over_n": round(float(t) / x.n, 4)} for (f, _, d, _), x, k, t in zip(spec, graphs, kc, tr)]
    return {"samples_per_graph": args.study_samples, "gpu_seconds": a.elapsed_time(b) / 1e3,
            "generate_seconds": round(t_gen, 1), "rows": rows}


# ------------------------------------------------------------ random-access ceiling

def random_access_ceiling(torch, args):
    """Ceiling of the Wilson step's memory pattern on this device: random
    single-byte read-then-write pairs over a buffer far above L2
    (lap_probe_random_rw, independent pairs, no dependent chain) at three
    launch sizes; the best rate is what the sampler's walk steps/s are
    compared with."""
    from paper_2311_10290_gb300.probe import lap_probe_random_rw
    free, _ = torch.cuda.mem_get_info()
    nbytes = min(64 << 30, int(free * 0.5)) // 256 * 256
    buf = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    rows, rounds = [], 64
    for k in (8, 16, 32):
        blocks = sms * k
        lap_probe_random_rw(buf, blocks, 4, salt=1, stream=stream)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        lap_probe_random_rw(buf, blocks, rounds, salt=100 + k, stream=stream)
        b.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 1e3
        rows.append({"blocks": blocks, "threads_per_block": 256, "pairs": blocks * 256 * rounds * 4,
                     "ms": round(t * 1e3, 3), "pairs_per_s": blocks * 256 * rounds * 4 / t})
    del buf
    torch.cuda.empty_cache()
    best = max(rows, key=lambda r: r["pairs_per_s"])
    return {"buffer_gb": round(nbytes / 1e9, 1), "pairs_per_s": best["pairs_per_s"], "rows": rows,
            "note": "random 1-byte read + write pairs, 4 independent per thread and round, SplitMix64 addresses"}


# ------------------------------------------------------------ extra workloads

def extra_workload(torch, LapGraph, name, args, params):
    """Plain throughput (1 warm-up and 1 timed launch of `extra_samples`
    samples) on another single-graph workload, then the control variate
    against plain on it when a trained network is given."""
    from paper_2311_10290_gb300.lap import LAP_STAT_FALLBACKS, LAP_STAT_LAST_KERNEL, lap_counts
    t0 = time.perf_counter()
    g = load_graph(name)
    t_gen = time.perf_counter() - t0
    free, _ = torch.cuda.mem_get_info()
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=int(free * args.ws_frac))
    try:
        v = G.set_root()
        B = args.extra_samples
        G.sample(B, args.seed)
        G.kemeny()
        _, c2a, sa = lap_counts(G.h, g.n)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        G.sample(B, args.seed)
        ev[1].record()
        G.ecc()
        kc = G.kemeny()
        ev[2].record()
        torch.cuda.synchronize()
        _, c2b, sb = lap_counts(G.h, g.n)
        wilson = int(sb[1]) - int(sa[1])
        uwalk = int(c2b.sum()) - int(c2a.sum())
        piwalk = int(sb[2]) - int(sa[2])
        t_kernel = ev[0].elapsed_time(ev[1]) / 1e3
        t_step = ev[0].elapsed_time(ev[2]) / 1e3
        alg = BYTES_WILSON_STEP * wilson + BYTES_TREE_INSERT * (g.n - 1) * B + BYTES_WALK_STEP * (uwalk + piwalk)
        peak, _ = peaks()
        res = {"workload": g.name, "n": g.n, "arcs": g.arcs, "root": v, "max_degree": int(np.diff(g.row_ptr).max()),
               "samples_per_step": B, "ms_per_step": t_step * 1e3, "value": (wilson + uwalk + piwalk) / t_step,
               "unit": "walk steps/s",
               "walk_steps": {"wilson": wilson, "uniform_walk": uwalk, "pi_walk": piwalk,
                              "wilson_steps_per_node_per_sample": wilson / B / g.n},
               "roofline": {"bound": "hbm", "achieved": alg / t_kernel / 1e9, "peak": peak, "unit": "GB/s",
                            "frac": alg / t_kernel / 1e9 / peak,
                            "traffic": measured_traffic(KERNEL_NAMES[G.stat(LAP_STAT_LAST_KERNEL)], wilson),
                            "traffic_note": "per launch, scaled from a small-case ncu capture by Wilson steps"},
               "kernel": KERNEL_NAMES[G.stat(LAP_STAT_LAST_KERNEL)], "fallbacks": G.stat(LAP_STAT_FALLBACKS),
               "kemeny_estimate": kc, "slots": G.slots, "generate_seconds": round(t_gen, 1)}
    finally:
        G.close()
    if params is not None:
        note("control variate: CV vs plain on %s" % g.name)
        res["cv_vs_plain"] = cv_measurement(torch, LapGraph, g, v, params, B, 4)
    return res


# ------------------------------------------------------------ uneven batch

def batched_measurement(torch, args):
    """Uneven batch: graphs of the recipe in inputs.batch_spec (ER, BA, R-MAT;
    n log-uniform in [1e3, 1e6]; average degree in [4, 32]; own root each),
    all sampled in one persistent CUDA-graph launch with autotuned lanes and
    claim size.  Times one run of `batched_samples` samples per graph after a
    warm-up run of 1/16 of them."""
    from paper_2311_10290_gb300 import inputs
    from paper_2311_10290_gb300.lap import LAP_BOPT_ORDER, LAP_BSTAT_CLAIM, LAP_BSTAT_LANES, LAP_BSTAT_RERUNS, LapBatch
    t0 = time.perf_counter()
    spec = inputs.batch_spec(count=args.batched_graphs, n_hi=args.batched_nmax)
    graphs = inputs.batch_graphs(spec)
    t_gen = time.perf_counter() - t0
    k, seed = args.batched_samples, args.seed
    t0 = time.perf_counter()
    B = LapBatch([(g.row_ptr, g.col) for g in graphs],
                 workspace_bytes=int(args.batched_ws_gb * 1e9) if args.batched_ws_gb > 0 else None)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    orders = [int(x) for x in args.batched_orders.split(",") if x.strip()]
    runs = []
    try:
        t0 = time.perf_counter()
        B.set_option(LAP_BOPT_ORDER, orders[0])
        table = B.autotune(k, seed)
        t_tune = time.perf_counter() - t0
        for order in orders:
            B.set_option(LAP_BOPT_ORDER, order)
            B.run(max(1, k // 16), seed + 1)            # warm-up (own CUDA graph)
            B.sync()
            torch.cuda.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record()
            B.run(k, seed)
            ev[1].record()
            B.sync()
            ev[2].record()
            torch.cuda.synchronize()
            done = B.completion()
            runs.append({"order": ["largest first", "smallest first", "given"][order],
                         "seconds": ev[0].elapsed_time(ev[2]) / 1e3,
                         "launch_seconds": ev[0].elapsed_time(ev[1]) / 1e3,
                         "completion_seconds": {"p50": float(np.percentile(done, 50)),
                                                "p99": float(np.percentile(done, 99)),
                                                "max": float(done.max()), "min": float(done.min())},
                         "reruns": B.stat(LAP_BSTAT_RERUNS)})
        kc = B.kemeny()
        wilson = uwalk = piwalk = inserts = 0
        for j, g in enumerate(graphs):
            _, c2, sums = B.counts(j)
            wilson += int(sums[1])
            piwalk += int(sums[2])
            uwalk += int(c2.sum(dtype=np.uint64))
            inserts += (g.n - 1) * k
        steps = wilson + uwalk + piwalk
        alg_bytes = BYTES_WILSON_STEP * wilson + BYTES_TREE_INSERT * inserts + BYTES_WALK_STEP * (uwalk + piwalk)
        peak, peak_kind = peaks()
        for r in runs:
            r["value"] = steps / r["seconds"]
            r["roofline_frac"] = alg_bytes / r["launch_seconds"] / 1e9 / peak
        best = max(runs, key=lambda r: r["value"])
        t_total, t_launch = best["seconds"], best["launch_seconds"]
        achieved = alg_bytes / t_launch / 1e9
        res = {
            "workload": "%d uneven graphs (ER/BA/R-MAT by seed mod 3, n log-uniform in [1e3, %.0e], average degree "
                        "uniform in [4, 32], seeds 0..%d; root = each graph's max-degree node)"
                        % (len(graphs), args.batched_nmax, len(graphs) - 1),
            "graphs": len(graphs), "total_nodes": int(sum(g.n for g in graphs)),
            "total_arcs": int(sum(g.arcs for g in graphs)), "largest_n": int(max(g.n for g in graphs)),
            "samples_per_graph": k, "seconds": t_total, "launch_seconds": t_launch,
            "walk_steps": {"wilson": wilson, "uniform_walk": uwalk, "pi_walk": piwalk},
            "value": steps / t_total, "unit": "walk steps/s",
            "completion_seconds": best["completion_seconds"], "order": best["order"], "runs": runs,
            "lanes": B.stat(LAP_BSTAT_LANES), "claim": B.stat(LAP_BSTAT_CLAIM), "reruns": best["reruns"],
            "autotune": [{"lanes": a, "claim": c, "walk_steps_per_s": round(r, 1)} for a, c, r in table],
            "autotune_seconds": round(t_tune, 2), "generate_seconds": round(t_gen, 2),
            "create_seconds": round(t_create, 2),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "kernel": "lewalk_batch_kernel (+ batched finalize, in one CUDA graph)",
                         "peak_kind": peak_kind},
            "kemeny_first_graphs": [round(float(x), 3) for x in kc[:4]],
            "note": "seconds: CUDA graph launch (resets, persistent sampler, finalize of every graph) to results "
                    "ready, re-runs of withdrawn samples included; completion: from the sampler's start to each "
                    "graph's last sample; top-level value/completion: the faster of `runs` (same samples, same "
                    "counts: only the unit order differs)",
        }
    finally:
        B.close()
    return res


# ------------------------------------------------------------ ours

def run_ours(args, rank, world):
    import torch
    from paper_2311_10290_gb300.lap import LAP_OPT_CURSOR, LapGraph, lap_counts
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    g = load_graph(args.workload)
    free, _ = torch.cuda.mem_get_info()
    ws = int(free * args.ws_frac)
    if args.ws_gb > 0:
        ws = min(ws, int(args.ws_gb * 1e9))
    G = LapGraph(g.row_ptr, g.col, workspace_bytes=ws)
    from paper_2311_10290_gb300.lap import LAP_OPT_KERNEL, LAP_OPT_WALKERS, LAP_STAT_KERNEL
    if args.kernel:
        G.set_option(LAP_OPT_KERNEL, args.kernel)
        G.set_option(LAP_OPT_WALKERS, args.walkers)
    v = G.set_root()
    kernel_name = KERNEL_NAMES[G.stat(LAP_STAT_KERNEL)]
    B = args.batch
    total_steps = args.warmup + args.steps
    from paper_2311_10290_gb300.shard import allreduce_counts, id_range
    first_id, _ = id_range(rank, world, world * total_steps * B)
    G.set_option(LAP_OPT_CURSOR, first_id)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # larger than the 126 MB L2
    out = torch.empty(g.n, dtype=torch.float64, device="cuda")

    def step():
        G.sample(B, args.seed)
        G.ecc(out)                      # finalize on device (ECC for every node)
        return G.kemeny()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    from paper_2311_10290_gb300.lap import LAP_STAT_LAST_KERNEL
    kernel_name = KERNEL_NAMES[G.stat(LAP_STAT_LAST_KERNEL)]
    c1a, c2a, sa = lap_counts(G.h, g.n)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with Clocks(dev) as clk:
        for k in range(args.steps):
            flush.zero_()                # L2 flush between timed steps (outside the events)
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            ev[k][0].record()
            G.sample(B, args.seed)
            ev[k][1].record()
            G.ecc(out)
            G.kemeny()
            ev[k][2].record()
            torch.cuda.synchronize()
    c1b, c2b, sb = lap_counts(G.h, g.n)
    merged = None
    if world > 1:
        # The one exchange step: sum the integer counts of all ranks, then
        # finalize the totals on rank 0 (outside the timed region).
        t0 = time.perf_counter()
        tot = allreduce_counts(torch.from_numpy(c1b.view(np.int64).copy()).cuda(),
                               torch.from_numpy(c2b.view(np.int64).copy()).cuda(),
                               torch.from_numpy(sb[:3].view(np.int64).copy()).cuda())
        if rank == 0:
            G.set_counts(*tot)
            merged = {"samples": int(tot[2][0].item()), "kemeny": G.kemeny(),
                      "ecc_mean": float(np.mean(G.ecc())), "exchange_seconds": time.perf_counter() - t0,
                      "exchange_bytes": 16 * g.n + 24}
    step_ms = [a.elapsed_time(c) for a, _, c in ev]
    kern_ms = [a.elapsed_time(b) for a, b, _ in ev]
    t_total = sum(step_ms) / 1e3
    wilson = int(sb[1]) - int(sa[1])
    uwalk = int(c2b.sum()) - int(c2a.sum())
    piwalk = int(sb[2]) - int(sa[2])
    samples = int(sb[0]) - int(sa[0])
    walk_steps = wilson + uwalk + piwalk
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([t_total], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        w = torch.tensor([walk_steps], dtype=torch.int64, device="cuda")
        dist.all_reduce(w)
        t_total, walk_steps_all = float(t.item()), int(w.item())
    else:
        walk_steps_all = walk_steps
    value = walk_steps_all / t_total
    kernel_s = sum(kern_ms) / 1e3 / args.steps
    alg_bytes = (BYTES_WILSON_STEP * wilson + BYTES_TREE_INSERT * (g.n - 1) * samples +
                 BYTES_WALK_STEP * (uwalk + piwalk)) / args.steps
    peak, peak_kind = peaks()
    achieved = alg_bytes / kernel_s / 1e9
    traffic = measured_traffic(kernel_name, wilson / args.steps)
    res = {
        "metric": HEADLINE_METRIC, "value": value, "unit": "walk steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64 counts, f64 finalize", "data": "synthetic",
        "config": {"workload": g.name + " (Barabasi-Albert n=1e6, m=5; root = max-degree node)"
                   if args.workload == "ba_1m" else g.name,
                   "n": g.n, "arcs": g.arcs, "root": v, "samples_per_step": B,
                   "samples_timed": samples * world, "slots": G.slots,
                   "workspace_gb": round(G.workspace.numel() / 1e9, 1),
                   "kernel": kernel_name,
                   "l2": "256 MB buffer written between timed steps (outside the events); "
                         "Wilson state working set far above L2",
                   "parallelism": "sample ids sharded over %d GPU(s)" % world},
        "walk_steps": {"wilson": wilson, "uniform_walk": uwalk, "pi_walk": piwalk,
                       "wilson_steps_per_node_per_sample": wilson / max(1, samples) / g.n},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": float(traffic) if traffic else None,
                     "traffic_note": "per launch, scaled from a small-case ncu capture by Wilson steps (profiles/)",
                     "kernel": kernel_name.split()[0], "kernel_ms": kernel_s * 1e3,
                     "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind},
        "gpu_launches": args.steps * 7,
    }
    if merged:
        res["merged_estimate"] = merged
    res["clocks"] = clk.summary()
    G.close()
    del flush, out
    torch.cuda.empty_cache()
    if rank == 0 and args.ceiling_probe:
        note("random-access ceiling probe")
        c = random_access_ceiling(torch, args)
        c["sampler_walk_steps_per_s"] = walk_steps / (kernel_s * args.steps)
        c["sampler_frac_of_ceiling"] = c["sampler_walk_steps_per_s"] / c["pairs_per_s"]
        res["random_access_ceiling"] = c
    # End to end through the C ABI with host buffers: each step copies the CSR
    # from pinned host memory (graph create), samples, finalizes and reads the
    # ECC vector and Kemeny's constant back to the host.
    if args.e2e_steps > 0:
        note("end to end through host buffers")
        res["e2e"] = run_e2e(args, g, torch, LapGraph, rank, world)
    if rank == 0 and not args.no_cpu and world == 1:
        note("CPU oracle baseline")
        res["cpu_baseline"] = cpu_oracle_rate(g, v, args.seed, args.cpu_seconds)
    if rank == 0 and not args.no_tta:
        note("time to accuracy (plain)")
        res["time_to_accuracy"] = time_to_accuracy(torch, LapGraph)
        if not args.no_cpu and world == 1 and res["time_to_accuracy"].get("omega"):
            note("time to accuracy: the CPU oracle at the same omega")
            res["time_to_accuracy"]["cpu_oracle"] = cpu_time_to_accuracy(res["time_to_accuracy"]["omega"])
    params = None
    if rank == 0 and args.cv_graphs > 0:
        note("control variate: training data and training")
        params, info = cv_train(torch, LapGraph, args.cv_graphs)
        note("control variate: MLP kernels (tcgen05 and mma.sync)")
        info["mlp_kernels"] = mlp_kernel_timing(torch)
        note("control variate: what the network learned (held-out graphs)")
        info["diagnostics"] = cv_diagnostics(torch, LapGraph, params)
        note("control variate: CV vs plain on %s" % g.name)
        info["graphs"] = [cv_measurement(torch, LapGraph, g, v, params, args.cv_batch, 4)]
        if not args.no_tta:
            note("time to accuracy (CV)")
            info["time_to_accuracy_cv"] = time_to_accuracy(torch, LapGraph, params=params)
        res["cv_vs_plain"] = info
    if rank == 0 and args.tta_large and not args.no_tta:
        out = []
        for spec in [x for x in args.tta_large.split(",") if x.strip()]:
            parts = spec.split(":")
            name, om = parts[0], parts[1]
            forms = parts[2].split("+") if len(parts) > 2 else [f for f in args.tta_forms.split(",") if f.strip()]
            note("time to accuracy on %s (grid to %s samples)" % (name, om))
            g2 = g if name == args.workload else load_graph(name)
            v2 = int(np.argmax(np.diff(g2.row_ptr)))          # the library's root: max degree, smallest id
            exact = exact_parts(torch, LapGraph, g2, v2)
            r = time_to_accuracy_large(torch, LapGraph, g2, v2, exact, int(om), forms=forms, params=params,
                                       seeds=args.tta_seeds)
            r = {"workload": g2.name, "n": g2.n, "arcs": g2.arcs, "root": v2, "exact_solve": exact["info"], **r}
            if not args.no_cpu and world == 1:
                om_star = max([r[f].get("omega", r[f].get("omega_extrapolated", 0)) for f in forms if f in r] or [0])
                if om_star:
                    r["cpu_oracle"] = cpu_oracle_extrapolated(g2, v2, args.seed, om_star)
            out.append(r)
            del exact
            torch.cuda.empty_cache()
        res["time_to_accuracy_large"] = out
    if rank == 0 and args.paths > 0:
        note("loop-included paths against own draws")
        res["paths_vs_own_draws"] = paths_measurement(torch, LapGraph, g, v, args)
        if not args.no_tta:
            res["paths_vs_own_draws"]["time_to_accuracy_paths"] = time_to_accuracy(torch, LapGraph, paths=1)
    if rank == 0 and args.spantree_trees > 0:
        note("SpanTree estimators")
        res["spantree"] = spantree_measurement(torch, LapGraph, g, v, args)
        res["spantree"]["lewalk_samples_per_s"] = samples / max(t_total, 1e-9)
    if rank == 0 and args.landmark_roots > 0:
        note("landmark study: %d roots" % args.landmark_roots)
        res["landmark_study"] = landmark_study(torch, g if args.workload == "ba_1m" else load_graph("ba_1m"), args)
    if rank == 0 and args.kemeny_sweep > 0:
        note("Kemeny sweep over 1e6-node BA and ER graphs")
        res["kemeny_sweep"] = kemeny_sweep(torch, args)
    for name in [x for x in args.extra_workloads.split(",") if x.strip()]:
        if rank != 0:
            break
        note("extra workload %s" % name)
        res.setdefault("extra_workloads", []).append(
            extra_workload(torch, LapGraph, name, args, params if args.cv_graphs > 0 and args.extra_cv else None))
    if rank == 0 and args.batched_graphs > 0:
        note("uneven batch: %d graphs" % args.batched_graphs)
        res["batched"] = batched_measurement(torch, args)
    if rank == 0:
        note("done")
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return res


def run_e2e(args, g, torch, LapGraph, rank, world):
    rp = torch.from_numpy(g.row_ptr).pin_memory()
    cl = torch.from_numpy(g.col).pin_memory()
    ecc_host = torch.empty(g.n, dtype=torch.float64).pin_memory()
    B = args.batch
    from paper_2311_10290_gb300.lap import LAP_OPT_CURSOR, lap_counts
    free, _ = torch.cuda.mem_get_info()
    ws = int(free * args.ws_frac)
    times, steps_total = [], 0
    for k in range(args.e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        H = LapGraph(rp.numpy(), cl.numpy(), workspace_bytes=ws)
        H.set_root()
        H.set_option(LAP_OPT_CURSOR, (1 << 31) + (rank * args.e2e_steps + k) * B)
        H.sample(B, args.seed)
        H.ecc(ecc_host.numpy())
        H.kemeny()
        t1 = time.perf_counter()
        _, c2, s = lap_counts(H.h, g.n)
        H.close()
        times.append(t1 - t0)
        steps_total += int(s[1]) + int(c2.sum()) + int(s[2])
    t = float(np.sum(times))
    if world > 1:
        # Whole job: walk steps of all ranks over the slowest rank's time.
        import torch.distributed as dist
        tt = torch.tensor([t], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        st = torch.tensor([steps_total], dtype=torch.int64, device="cuda")
        dist.all_reduce(st)
        t, steps_total = float(tt.item()), int(st.item())
    return {"value": steps_total / t, "unit": "walk steps/s",
            "h2d_bytes_per_step": int(rp.numel() * 4 + cl.numel() * 4),
            "d2h_bytes_per_step": int(g.n * 8 + 8),
            "ms_per_step": 1e3 * t / len(times),
            "note": "graph create (H2D of the CSR, GPU validation, BFS) + sample + finalize + D2H of ECC and Kemeny"}


# ------------------------------------------------------------ reference (oracle)

def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle
    g = load_graph(args.workload)
    v = oracle.root_max_degree(g.row_ptr)
    cores = os.cpu_count() or 1
    # Size a step to a few seconds of host time.
    t0 = time.perf_counter()
    oracle.sample(g.row_ptr, g.col, v, args.seed, 0, 1)
    per = max(time.perf_counter() - t0, 1e-4)
    per_step = cores * max(1, min(64, int(4.0 / per)))
    times, steps = [], 0
    nxt = 1
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        c = oracle.sample_threads(g.row_ptr, g.col, v, args.seed, nxt, per_step, cores)
        ld, ec, kc = oracle.finalize(g.row_ptr, v, per_step, c.cnt1, c.cnt2, c.sum_y1, c.sum_y2)
        dt = time.perf_counter() - t0
        nxt += per_step
        if k >= args.warmup:
            times.append(dt)
            steps += c.sum_y1 + int(c.cnt2.sum()) + c.sum_y2
    t = float(np.sum(times))
    value = steps / t
    return {"impl": "reference", "metric": HEADLINE_METRIC, "value": value, "unit": "walk steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64 counts, f64 finalize", "data": "synthetic",
            "config": {"workload": g.name, "n": g.n, "arcs": g.arcs, "root": v, "samples_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "walk steps/s", "cores": cores, "kind": "oracle",
                             "sample": "%d samples per step on %d threads (bounded sample of the workload)" %
                                       (per_step, cores)},
            "e2e": {"value": value, "unit": "walk steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_ours(args, rank, world)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
