"""Thin Python binding of the C ABI in include/lap.h (argument marshalling only).

Every step of the sampling path runs in the CUDA library ``liblap.so``; this
module only converts arguments, lends torch-allocated device memory (the
Wilson-state workspace) and the current torch stream to the library, and
turns status codes into exceptions.  Importing it fails loudly when the
library has not been built: there is no CPU fallback.

Functions keep the C names (``lap_graph_create``, ``lap_set_root``,
``lap_sample``, ``lap_ecc``, ``lap_kemeny`` ...); :class:`LapGraph` bundles
them for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblap.so")

STATUS = {
    0: "LAP_OK", 1: "LAP_ERR_INVALID_ARG", 2: "LAP_ERR_BAD_CSR", 3: "LAP_ERR_NOT_SYMMETRIC",
    4: "LAP_ERR_SELF_LOOP", 5: "LAP_ERR_DISCONNECTED", 6: "LAP_ERR_TOO_LARGE", 7: "LAP_ERR_OOM",
    8: "LAP_ERR_NO_SAMPLES", 9: "LAP_ERR_STEP_LIMIT", 10: "LAP_ERR_CUDA", 11: "LAP_ERR_NO_ROOT",
}
LAP_OPT_STEP_LIMIT, LAP_OPT_SLOTS, LAP_OPT_BLOCK, LAP_OPT_CURSOR, LAP_OPT_KERNEL, LAP_OPT_STACK = 1, 2, 3, 4, 5, 6
LAP_OPT_PATHS = 7
LAP_OPT_PATH_START = 8
LAP_OPT_WALKERS = 9
LAP_STAT_SLOTS, LAP_STAT_KERNEL, LAP_STAT_FALLBACKS, LAP_STAT_LAST_KERNEL = 1, 2, 3, 4
LAP_MLP_PARAMS = 4866
LAP_MLP_TCGEN05, LAP_MLP_MMA_SYNC = 0, 1
LAP_BOPT_LANES, LAP_BOPT_CLAIM, LAP_BOPT_ORDER, LAP_BOPT_BLOCK, LAP_BOPT_STACK, LAP_BOPT_PATHS = 1, 2, 3, 4, 5, 6
LAP_BSTAT_LANES, LAP_BSTAT_CLAIM, LAP_BSTAT_UNITS, LAP_BSTAT_RERUNS, LAP_BSTAT_GRAPH_CAPTURES = 1, 2, 3, 4, 5


class LapError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status
        self.name = STATUS.get(status, str(status))


_lib = None


def library():
    """The loaded liblap.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("liblap.so is not built (run __graft_entry__.build() or "
                          "python paper_2311_10290_gb300/build.py); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "lap_version": (i32, []),
        "lap_graph_create": (i32, [i32, vp, vp, ctypes.c_int, ctypes.POINTER(vp)]),
        "lap_graph_destroy": (i32, [vp]),
        "lap_set_stream": (i32, [vp, vp]),
        "lap_set_option": (i32, [vp, i32, i64]),
        "lap_workspace_query": (i32, [vp, u64, ctypes.POINTER(u64)]),
        "lap_set_workspace": (i32, [vp, vp, u64]),
        "lap_set_root": (i32, [vp, i32, ctypes.POINTER(i32)]),
        "lap_sample": (i32, [vp, u64, u64]),
        "lap_sample_trace": (i32, [vp, u64, u64, vp, vp]),
        "lap_sync": (i32, [vp]),
        "lap_ecc": (i32, [vp, vp, ctypes.c_int]),
        "lap_ldiag": (i32, [vp, vp, ctypes.c_int]),
        "lap_kemeny": (i32, [vp, vp]),
        "lap_lv_row": (i32, [vp, vp, ctypes.c_int]),
        "lap_lv_solve": (i32, [vp, vp, vp, ctypes.c_int, ctypes.c_double, i32, ctypes.POINTER(i32),
                               ctypes.POINTER(ctypes.c_double)]),
        "lap_batch_set_path_start": (i32, [vp, i32, i32]),
        "lap_batch_lv_row": (i32, [vp, i32, vp, ctypes.c_int]),
        "lap_counts": (i32, [vp, vp, vp, vp, ctypes.c_int]),
        "lap_hops": (i32, [vp, vp, ctypes.c_int]),
        "lap_set_counts": (i32, [vp, vp, vp, vp, ctypes.c_int]),
        "lap_kirchhoff": (i32, [vp, vp]),
        "lap_spantree_sample": (i32, [vp, u64, u64]),
        "lap_spantree_sums": (i32, [vp, vp, vp, vp, ctypes.POINTER(u64), ctypes.c_int]),
        "lap_spantree_estimates": (i32, [vp, vp, vp, ctypes.c_int, vp]),
        "lap_rw_betweenness": (i32, [vp, vp, ctypes.c_int]),
        "lap_batch_kirchhoff": (i32, [vp, vp]),
        "lap_get_stat": (i32, [vp, i32, ctypes.POINTER(i64)]),
        "lap_graph_info": (i32, [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32)]),
        "lap_last_error": (ctypes.c_char_p, [vp]),
        "lap_sample_static": (i32, [i32, vp, vp, i32, u64, u64, u64, vp, vp, vp, vp]),
        "lap_features": (i32, [vp, vp]),
        "lap_hitting_walks": (i32, [vp, ctypes.c_uint32, u64, vp]),
        "lap_cv_set_potentials": (i32, [vp, vp, vp]),
        "lap_cv_targets": (i32, [vp, ctypes.c_uint32, u64, vp]),
        "lap_cv_potentials": (i32, [vp, vp, vp, vp]),
        "lap_cv_fit_betas": (i32, [vp, vp, vp, u64, u64, u64, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double)]),
        "lap_cv_sums": (i32, [vp, vp, vp, vp, ctypes.c_int]),
        "lap_cv_set_sums": (i32, [vp, vp, vp, vp, ctypes.c_int]),
        "lap_cv_estimates": (i32, [vp, ctypes.c_double, ctypes.c_double, vp, vp, ctypes.c_int, vp, vp]),
        "lap_sample_trace_cv": (i32, [vp, u64, u64, vp, vp, vp]),
        "lap_mlp_select": (i32, [i32]),
        "lap_mlp_forward": (i32, [vp, vp, i64, vp, vp]),
        "lap_mlp_loss_grad": (i32, [vp, vp, vp, i64, ctypes.c_float, ctypes.c_float, vp, vp, vp]),
        "lap_adamw": (i32, [vp, vp, vp, vp, i64, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                            ctypes.c_float, ctypes.c_float, vp]),
        "lap_static_scratch_bytes": (u64, []),
        "lap_static_last_error": (ctypes.c_char_p, []),
        "lap_batch_create": (i32, [i32, vp, vp, vp, vp, ctypes.POINTER(vp)]),
        "lap_batch_destroy": (i32, [vp]),
        "lap_batch_set_stream": (i32, [vp, vp]),
        "lap_batch_set_option": (i32, [vp, i32, i64]),
        "lap_batch_workspace_query": (i32, [vp, u64, ctypes.POINTER(u64)]),
        "lap_batch_set_workspace": (i32, [vp, vp, u64]),
        "lap_batch_autotune": (i32, [vp, u64, u64, ctypes.c_double, i32, vp, vp, vp, ctypes.POINTER(i32)]),
        "lap_batch_run": (i32, [vp, u64, u64]),
        "lap_batch_sync": (i32, [vp]),
        "lap_batch_ecc": (i32, [vp, vp, ctypes.c_int]),
        "lap_batch_ldiag": (i32, [vp, vp, ctypes.c_int]),
        "lap_batch_kemeny": (i32, [vp, vp]),
        "lap_batch_completion": (i32, [vp, vp]),
        "lap_batch_counts": (i32, [vp, i32, vp, vp, vp, ctypes.c_int]),
        "lap_batch_graph_info": (i32, [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                       ctypes.POINTER(i64)]),
        "lap_batch_stat": (i32, [vp, i32, ctypes.POINTER(i64)]),
        "lap_batch_schedule": (i32, [i32, vp, i32, u64, ctypes.c_uint32, vp, vp, u64, ctypes.POINTER(u64)]),
        "lap_batch_last_error": (ctypes.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status, handle=None):
    if status != 0:
        msg = library().lap_last_error(handle)
        raise LapError(status, msg.decode() if msg else "")


def _host_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _is_torch(x):
    return type(x).__module__.startswith("torch")


# ------------------------------------------------------------ C-named calls

def lap_version():
    return library().lap_version()


def lap_last_error(h=None):
    m = library().lap_last_error(h)
    return m.decode() if m else ""


def lap_graph_create(n, row_ptr, col_idx):
    """row_ptr/col_idx: int32 numpy arrays (host) or int32 CUDA torch tensors."""
    if _is_torch(row_ptr):
        assert row_ptr.is_cuda and col_idx.is_cuda and row_ptr.dtype == col_idx.dtype
        ptrs = (ctypes.c_void_p(row_ptr.data_ptr()), ctypes.c_void_p(col_idx.data_ptr()), 1)
    else:
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        cl = np.ascontiguousarray(col_idx, dtype=np.int32)
        ptrs = (_host_ptr(rp), _host_ptr(cl), 0)
    h = ctypes.c_void_p()
    _check(library().lap_graph_create(int(n), ptrs[0], ptrs[1], ptrs[2], ctypes.byref(h)))
    return h


def lap_graph_destroy(h):
    _check(library().lap_graph_destroy(h))


def lap_set_stream(h, stream_ptr):
    _check(library().lap_set_stream(h, ctypes.c_void_p(stream_ptr)), h)


def lap_set_option(h, option, value):
    _check(library().lap_set_option(h, int(option), int(value)), h)


def lap_workspace_query(h, slots):
    b = ctypes.c_uint64()
    _check(library().lap_workspace_query(h, int(slots), ctypes.byref(b)), h)
    return b.value


def lap_set_workspace(h, dev_ptr, nbytes):
    _check(library().lap_set_workspace(h, ctypes.c_void_p(dev_ptr), int(nbytes)), h)


def lap_set_root(h, v=-1):
    r = ctypes.c_int32()
    _check(library().lap_set_root(h, int(v), ctypes.byref(r)), h)
    return r.value


def lap_sample(h, n_samples, seed):
    _check(library().lap_sample(h, int(n_samples), int(seed)), h)


def lap_sample_trace(h, n_samples, seed, y1_dev, y2_dev):
    """y1_dev, y2_dev: uint64 (int64) CUDA torch tensors of n_samples entries."""
    _check(library().lap_sample_trace(h, int(n_samples), int(seed), ctypes.c_void_p(y1_dev.data_ptr()),
                                      ctypes.c_void_p(y2_dev.data_ptr())), h)


def lap_sync(h):
    _check(library().lap_sync(h), h)


def _out(h, fn, n, dtype, out):
    if out is None:
        out = np.empty(n, dtype=dtype)
    if _is_torch(out):
        _check(fn(h, ctypes.c_void_p(out.data_ptr()), 1), h)
    else:
        _check(fn(h, _host_ptr(out), 0), h)
    return out


def lap_ecc(h, n, out=None):
    return _out(h, library().lap_ecc, n, np.float64, out)


def lap_ldiag(h, n, out=None):
    return _out(h, library().lap_ldiag, n, np.float64, out)


def lap_lv_row(h, n, out=None):
    return _out(h, library().lap_lv_row, n, np.float64, out)


def lap_lv_solve(h, n, b, rtol=1e-12, maxiter=100000, out=None):
    """x = L_v^{-1} b; b a float64 numpy array (host) or CUDA tensor (device);
    returns (x, iterations, residual)."""
    it, res = ctypes.c_int32(0), ctypes.c_double(0.0)
    if _is_torch(b):
        x = out if out is not None else b.new_empty(n)
        _check(library().lap_lv_solve(h, _dp(b), _dp(x), 1, float(rtol), int(maxiter), ctypes.byref(it),
                                      ctypes.byref(res)), h)
    else:
        bb = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(n) if out is None else out
        _check(library().lap_lv_solve(h, _host_ptr(bb), _host_ptr(x), 0, float(rtol), int(maxiter),
                                      ctypes.byref(it), ctypes.byref(res)), h)
    return x, it.value, res.value


def lap_hops(h, n, out=None):
    return _out(h, library().lap_hops, n, np.int32, out)


def lap_kemeny(h):
    x = np.zeros(1, dtype=np.float64)
    _check(library().lap_kemeny(h, _host_ptr(x)), h)
    return float(x[0])


def lap_counts(h, n, per_node=True):
    """(cnt1, cnt2, sums) as host uint64 arrays; per_node=False reads only sums."""
    c1 = np.zeros(n, dtype=np.uint64) if per_node else None
    c2 = np.zeros(n, dtype=np.uint64) if per_node else None
    s = np.zeros(4, dtype=np.uint64)
    _check(library().lap_counts(h, None if c1 is None else _host_ptr(c1), None if c2 is None else _host_ptr(c2),
                                _host_ptr(s), 0), h)
    return c1, c2, s


def lap_spantree_sample(h, n_samples, seed):
    _check(library().lap_spantree_sample(h, int(n_samples), int(seed)), h)


def lap_spantree_sums(h, n):
    """Host int64 (x1, x2, x2d) sums and the number of trees."""
    x1, x2, x2d = (np.zeros(n, dtype=np.int64) for _ in range(3))
    om = ctypes.c_uint64()
    _check(library().lap_spantree_sums(h, _host_ptr(x1), _host_ptr(x2), _host_ptr(x2d), ctypes.byref(om), 0), h)
    return x1, x2, x2d, om.value


def lap_spantree_estimates(h, n):
    """Host (ldiag, ecc) and Kemeny's constant of the SpanTree estimators."""
    ld = np.zeros(n)
    ec = np.zeros(n)
    kc = np.zeros(1)
    _check(library().lap_spantree_estimates(h, _host_ptr(ld), _host_ptr(ec), 0, _host_ptr(kc)), h)
    return ld, ec, float(kc[0])


def lap_kirchhoff(h):
    out = np.zeros(1)
    _check(library().lap_kirchhoff(h, _host_ptr(out)), h)
    return float(out[0])


def lap_rw_betweenness(h, n, out=None):
    return _out(h, library().lap_rw_betweenness, n, np.float64, out)


def lap_set_counts(h, cnt1, cnt2, sums):
    """Replaces the handle's counts: cnt1, cnt2 uint64/int64 [n] and sums
    {omega, sum Y1, sum Y2}, all host numpy arrays or all CUDA tensors."""
    if _is_torch(cnt1):
        _check(library().lap_set_counts(h, _dp(cnt1), _dp(cnt2), _dp(sums), 1), h)
        return
    c1 = np.ascontiguousarray(cnt1, dtype=np.uint64)
    c2 = np.ascontiguousarray(cnt2, dtype=np.uint64)
    s3 = np.ascontiguousarray(np.asarray(sums)[:3], dtype=np.uint64)
    _check(library().lap_set_counts(h, _host_ptr(c1), _host_ptr(c2), _host_ptr(s3), 0), h)


def lap_get_stat(h, stat):
    x = ctypes.c_int64()
    _check(library().lap_get_stat(h, int(stat), ctypes.byref(x)), h)
    return x.value


def lap_graph_info(h):
    n, a, r = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32()
    _check(library().lap_graph_info(h, ctypes.byref(n), ctypes.byref(a), ctypes.byref(r)), h)
    return n.value, a.value, r.value


def lap_static_scratch_bytes():
    return library().lap_static_scratch_bytes()


def lap_static_last_error():
    m = library().lap_static_last_error()
    return m.decode() if m else ""


def lap_sample_static(n, row_ptr, col_idx, root, seed, first_id, n_samples, cnt1, cnt2, sums2, stream=0):
    """Allocation-free sampler (see include/lap.h).  row_ptr/col_idx: int32
    CUDA tensors; cnt1/cnt2: 64-bit CUDA tensors of n entries; sums2: 64-bit
    CUDA tensor of 2 entries; stream: a cudaStream_t as an integer."""
    st = library().lap_sample_static(int(n), ctypes.c_void_p(row_ptr.data_ptr()), ctypes.c_void_p(col_idx.data_ptr()),
                                     int(root), int(seed), int(first_id), int(n_samples),
                                     ctypes.c_void_p(cnt1.data_ptr()), ctypes.c_void_p(cnt2.data_ptr()),
                                     ctypes.c_void_p(sums2.data_ptr()), ctypes.c_void_p(int(stream)))
    if st != 0:
        raise LapError(st, lap_static_last_error())


def _dp(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def lap_features(h, feat_dev):
    """feat_dev: float32 CUDA tensor [n, 8]."""
    _check(library().lap_features(h, _dp(feat_dev)), h)


def lap_hitting_walks(h, reps, seed, sums_dev):
    """sums_dev: 64-bit CUDA tensor [n], overwritten with total walk lengths."""
    _check(library().lap_hitting_walks(h, int(reps), int(seed), _dp(sums_dev)), h)


def lap_cv_set_potentials(h, phi1_dev=None, phi2_dev=None):
    """phi1_dev, phi2_dev: float64 CUDA tensors [n] or None."""
    _check(library().lap_cv_set_potentials(h, _dp(phi1_dev), _dp(phi2_dev)), h)


def lap_cv_targets(h, reps, seed, targets_dev):
    """targets_dev: float32 CUDA tensor [n, 2] (overwritten)."""
    _check(library().lap_cv_targets(h, int(reps), int(seed), _dp(targets_dev)), h)


def lap_cv_potentials(h, y_dev, phi1_dev=None, phi2_dev=None):
    """y_dev: float32 CUDA tensor [n, 2]; phi1_dev, phi2_dev: float64 CUDA tensors [n] or None."""
    _check(library().lap_cv_potentials(h, _dp(y_dev), _dp(phi1_dev), _dp(phi2_dev)), h)


def lap_cv_fit_betas(h, phi1_dev, phi2_dev, seed, first_id, pilot, batches):
    """Returns (beta1, beta2)."""
    b1, b2 = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(library().lap_cv_fit_betas(h, _dp(phi1_dev), _dp(phi2_dev), int(seed), int(first_id), int(pilot),
                                      int(batches), ctypes.byref(b1), ctypes.byref(b2)), h)
    return b1.value, b2.value


def lap_cv_sums(h, n):
    a1, a2, p2 = (np.zeros(n, dtype=np.int64) for _ in range(3))
    _check(library().lap_cv_sums(h, _host_ptr(a1), _host_ptr(a2), _host_ptr(p2), 0), h)
    return a1, a2, p2


def lap_cv_set_sums(h, a1, a2, p2):
    """a1, a2, p2: int64 arrays (numpy: host; torch CUDA tensors: device)."""
    if _is_torch(a1):
        _check(library().lap_cv_set_sums(h, _dp(a1), _dp(a2), _dp(p2), 1), h)
    else:
        a = [np.ascontiguousarray(x, dtype=np.int64) for x in (a1, a2, p2)]
        _check(library().lap_cv_set_sums(h, _host_ptr(a[0]), _host_ptr(a[1]), _host_ptr(a[2]), 0), h)


def lap_cv_estimates(h, n, beta1, beta2, ecc_out=None):
    """Returns (ldiag, ecc, kemeny, m2_total) of the control-variate estimators.
    With a float64 CUDA tensor `ecc_out` the ECC goes there (device) and
    ldiag is not read: returns (None, ecc_out, kemeny, m2_total)."""
    if ecc_out is not None:
        kc = np.zeros(1)
        m2 = np.zeros(1)
        _check(library().lap_cv_estimates(h, float(beta1), float(beta2), None, _dp(ecc_out), 1,
                                          _host_ptr(kc), _host_ptr(m2)), h)
        return None, ecc_out, float(kc[0]), float(m2[0])
    ld = np.zeros(n)
    ec = np.zeros(n)
    kc = np.zeros(1)
    m2 = np.zeros(1)
    _check(library().lap_cv_estimates(h, float(beta1), float(beta2), _host_ptr(ld), _host_ptr(ec), 0,
                                      _host_ptr(kc), _host_ptr(m2)), h)
    return ld, ec, float(kc[0]), float(m2[0])


def lap_sample_trace_cv(h, n_samples, seed, y1_dev, y2_dev, m2_dev):
    _check(library().lap_sample_trace_cv(h, int(n_samples), int(seed), _dp(y1_dev), _dp(y2_dev), _dp(m2_dev)), h)


def lap_mlp_select(kernel):
    _check(library().lap_mlp_select(int(kernel)))


def lap_mlp_forward(params_dev, x_dev, rows, y_dev, stream=0):
    _check(library().lap_mlp_forward(_dp(params_dev), _dp(x_dev), int(rows), _dp(y_dev), ctypes.c_void_p(int(stream))))


def lap_mlp_loss_grad(params_dev, x_dev, t_dev, rows, w0, w1, grad_dev, loss_dev, stream=0):
    _check(library().lap_mlp_loss_grad(_dp(params_dev), _dp(x_dev), _dp(t_dev), int(rows), float(w0), float(w1),
                                       _dp(grad_dev), _dp(loss_dev), ctypes.c_void_p(int(stream))))


def lap_adamw(params_dev, m_dev, v_dev, grad_dev, count, step, lr, beta1=0.9, beta2=0.999, eps=1e-8,
              weight_decay=0.0, stream=0):
    _check(library().lap_adamw(_dp(params_dev), _dp(m_dev), _dp(v_dev), _dp(grad_dev), int(count), int(step),
                               float(lr), float(beta1), float(beta2), float(eps), float(weight_decay),
                               ctypes.c_void_p(int(stream))))


# ------------------------------------------------------------ batches (include/lap_batch.h)

def _bcheck(status, handle=None):
    if status != 0:
        msg = library().lap_batch_last_error(handle)
        raise LapError(status, msg.decode() if msg else "")


def lap_batch_create(graphs, roots=None):
    """graphs: sequence of (row_ptr, col) host int32 arrays; roots: int32 per
    graph (< 0: highest degree) or None.  Returns the handle."""
    # The same array objects map to the same host pointers, which the library
    # turns into one shared device copy (one graph sampled from many roots).
    conv = {}

    def c32(a):
        key = id(a)
        if key not in conv:
            conv[key] = (a, np.ascontiguousarray(a, dtype=np.int32))
        return conv[key][1]

    rps = [c32(r) for r, _ in graphs]
    cols = [c32(c) for _, c in graphs]
    ns = np.array([r.size - 1 for r in rps], dtype=np.int32)
    rp_ptrs = (ctypes.c_void_p * len(rps))(*[r.ctypes.data for r in rps])
    col_ptrs = (ctypes.c_void_p * len(cols))(*[c.ctypes.data for c in cols])
    rt = None if roots is None else np.ascontiguousarray(roots, dtype=np.int32)
    h = ctypes.c_void_p()
    _bcheck(library().lap_batch_create(len(rps), _host_ptr(ns), rp_ptrs, col_ptrs,
                                       None if rt is None else _host_ptr(rt), ctypes.byref(h)))
    return h


def lap_batch_destroy(h):
    _bcheck(library().lap_batch_destroy(h), h)


def lap_batch_set_stream(h, stream_ptr):
    _bcheck(library().lap_batch_set_stream(h, ctypes.c_void_p(int(stream_ptr))), h)


def lap_batch_set_option(h, option, value):
    _bcheck(library().lap_batch_set_option(h, int(option), int(value)), h)


def lap_batch_workspace_query(h, lanes):
    out = ctypes.c_uint64()
    _bcheck(library().lap_batch_workspace_query(h, int(lanes), ctypes.byref(out)), h)
    return out.value


def lap_batch_set_workspace(h, dev_ptr, nbytes):
    _bcheck(library().lap_batch_set_workspace(h, ctypes.c_void_p(int(dev_ptr)), int(nbytes)), h)


def lap_batch_autotune(h, samples_per_graph, seed, window_ms=300.0, max_trials=16):
    """Returns the probe table [(lanes, claim, steps/s), ...]."""
    lanes = np.zeros(max_trials, dtype=np.int64)
    claim = np.zeros(max_trials, dtype=np.int32)
    sps = np.zeros(max_trials, dtype=np.float64)
    rows = ctypes.c_int32()
    _bcheck(library().lap_batch_autotune(h, int(samples_per_graph), int(seed), float(window_ms), max_trials,
                                         _host_ptr(lanes), _host_ptr(claim), _host_ptr(sps), ctypes.byref(rows)), h)
    k = min(rows.value, max_trials)
    return [(int(lanes[j]), int(claim[j]), float(sps[j])) for j in range(k)]


def lap_batch_run(h, samples_per_graph, seed):
    _bcheck(library().lap_batch_run(h, int(samples_per_graph), int(seed)), h)


def lap_batch_sync(h):
    _bcheck(library().lap_batch_sync(h), h)


def lap_batch_ecc(h, total_n, out=None):
    if out is not None:
        _bcheck(library().lap_batch_ecc(h, _dp(out), 1), h)
        return out
    a = np.zeros(total_n)
    _bcheck(library().lap_batch_ecc(h, _host_ptr(a), 0), h)
    return a


def lap_batch_ldiag(h, total_n, out=None):
    if out is not None:
        _bcheck(library().lap_batch_ldiag(h, _dp(out), 1), h)
        return out
    a = np.zeros(total_n)
    _bcheck(library().lap_batch_ldiag(h, _host_ptr(a), 0), h)
    return a


def lap_batch_kemeny(h, n_graphs):
    a = np.zeros(n_graphs)
    _bcheck(library().lap_batch_kemeny(h, _host_ptr(a)), h)
    return a


def lap_batch_kirchhoff(h, n_graphs):
    a = np.zeros(n_graphs)
    _bcheck(library().lap_batch_kirchhoff(h, _host_ptr(a)), h)
    return a


def lap_batch_completion(h, n_graphs):
    a = np.zeros(n_graphs)
    _bcheck(library().lap_batch_completion(h, _host_ptr(a)), h)
    return a


def lap_batch_set_path_start(h, graph, start):
    _bcheck(library().lap_batch_set_path_start(h, int(graph), int(start)), h)


def lap_batch_lv_row(h, graph, n, out=None):
    if out is not None and _is_torch(out):
        _bcheck(library().lap_batch_lv_row(h, int(graph), _dp(out), 1), h)
        return out
    a = np.zeros(n) if out is None else out
    _bcheck(library().lap_batch_lv_row(h, int(graph), _host_ptr(a), 0), h)
    return a


def lap_batch_counts(h, graph, n, per_node=True):
    """Host (cnt1, cnt2, sums {omega, sum Y1, sum Y2, seed}) of one graph;
    per_node=False reads only the sums."""
    c1 = np.zeros(n, dtype=np.uint64) if per_node else None
    c2 = np.zeros(n, dtype=np.uint64) if per_node else None
    sums = np.zeros(4, dtype=np.uint64)
    _bcheck(library().lap_batch_counts(h, int(graph), None if c1 is None else _host_ptr(c1),
                                       None if c2 is None else _host_ptr(c2), _host_ptr(sums), 0), h)
    return c1, c2, sums


def lap_batch_graph_info(h, graph):
    n, arcs, root, off = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
    _bcheck(library().lap_batch_graph_info(h, int(graph), ctypes.byref(n), ctypes.byref(arcs), ctypes.byref(root),
                                           ctypes.byref(off)), h)
    return n.value, arcs.value, root.value, off.value


def lap_batch_stat(h, which):
    out = ctypes.c_int64()
    _bcheck(library().lap_batch_stat(h, int(which), ctypes.byref(out)), h)
    return out.value


def lap_batch_schedule(n, order, samples, claim):
    """Host-only: the work-unit queue as (graph, first sample) arrays."""
    ns = np.ascontiguousarray(n, dtype=np.int32)
    count = ctypes.c_uint64()
    library().lap_batch_schedule(ns.size, _host_ptr(ns), int(order), int(samples), int(claim), None, None, 0,
                                 ctypes.byref(count))
    ug = np.zeros(max(1, count.value), dtype=np.uint32)
    uf = np.zeros(max(1, count.value), dtype=np.uint32)
    _bcheck(library().lap_batch_schedule(ns.size, _host_ptr(ns), int(order), int(samples), int(claim),
                                         _host_ptr(ug), _host_ptr(uf), ug.size, ctypes.byref(count)))
    return ug[:count.value], uf[:count.value]


def lap_batch_last_error(h=None):
    m = library().lap_batch_last_error(h)
    return m.decode() if m else ""


# ------------------------------------------------------------ convenience

class LapGraph:
    """A graph handle with a torch-allocated Wilson-state workspace.

    row_ptr/col: numpy int32 (host, copied in) or CUDA int32 torch tensors.
    workspace_bytes: bytes of device memory lent to the sampler (default: 60%
    of the free device memory, capped at what 152 SMs x 2048 lanes can use).
    """

    def __init__(self, row_ptr, col, workspace_bytes=None, stream=None):
        import torch
        self.n = int(len(row_ptr) - 1)
        self.row_ptr_host = row_ptr.cpu().numpy() if _is_torch(row_ptr) else np.asarray(row_ptr)
        self.col_host = col.cpu().numpy() if _is_torch(col) else np.asarray(col)
        self.h = lap_graph_create(self.n, row_ptr, col)
        self._torch = torch
        s = stream if stream is not None else torch.cuda.current_stream()
        lap_set_stream(self.h, s.cuda_stream)
        per_slot = 8 * self.n
        if workspace_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
            workspace_bytes = min(int(free * 0.6), per_slot * sms * 2048)
        workspace_bytes = max(per_slot, (int(workspace_bytes) // per_slot) * per_slot)
        self.workspace = torch.empty(workspace_bytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        lap_set_workspace(self.h, aligned, workspace_bytes)
        self.root = None

    @property
    def slots(self):
        """Samples in flight per launch with the current kernel and workspace."""
        return lap_get_stat(self.h, LAP_STAT_SLOTS)

    def stat(self, which):
        return lap_get_stat(self.h, which)

    def close(self):
        if self.h is not None:
            lap_graph_destroy(self.h)
            self.h = None
            self.workspace = None
            self._torch.cuda.empty_cache()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option, value):
        lap_set_option(self.h, option, value)

    def set_root(self, v=-1):
        self.root = lap_set_root(self.h, v)
        return self.root

    def sample(self, n_samples, seed):
        lap_sample(self.h, n_samples, seed)

    def sample_trace(self, n_samples, seed):
        """Returns per-sample (Y1, Y2) as int64 CUDA tensors (asynchronous)."""
        y1 = self._torch.zeros(n_samples, dtype=self._torch.int64, device="cuda")
        y2 = self._torch.zeros(n_samples, dtype=self._torch.int64, device="cuda")
        lap_sample_trace(self.h, n_samples, seed, y1, y2)
        return y1, y2

    def sync(self):
        lap_sync(self.h)

    def ecc(self, out=None):
        return lap_ecc(self.h, self.n, out)

    def ldiag(self, out=None):
        return lap_ldiag(self.h, self.n, out)

    def kemeny(self):
        return lap_kemeny(self.h)

    def lv_row(self, out=None):
        return lap_lv_row(self.h, self.n, out)

    def lv_solve(self, b, rtol=1e-12, maxiter=100000, out=None):
        return lap_lv_solve(self.h, self.n, b, rtol, maxiter, out)

    def counts(self, per_node=True):
        return lap_counts(self.h, self.n, per_node)

    def hops(self, out=None):
        return lap_hops(self.h, self.n, out)

    def kirchhoff(self):
        return lap_kirchhoff(self.h)

    def spantree_sample(self, n_samples, seed):
        lap_spantree_sample(self.h, n_samples, seed)

    def spantree_sums(self):
        return lap_spantree_sums(self.h, self.n)

    def spantree_estimates(self):
        return lap_spantree_estimates(self.h, self.n)

    def rw_betweenness(self, out=None):
        return lap_rw_betweenness(self.h, self.n, out)

    def set_counts(self, cnt1, cnt2, sums):
        lap_set_counts(self.h, cnt1, cnt2, sums)

    def features(self):
        f = self._torch.empty((self.n, 8), dtype=self._torch.float32, device="cuda")
        lap_features(self.h, f)
        return f

    def hitting_walks(self, reps, seed):
        out = self._torch.empty(self.n, dtype=self._torch.int64, device="cuda")
        lap_hitting_walks(self.h, reps, seed, out)
        return out

    def cv_set_potentials(self, phi1=None, phi2=None):
        lap_cv_set_potentials(self.h, phi1, phi2)

    def cv_targets(self, reps, seed):
        t = self._torch.empty((self.n, 2), dtype=self._torch.float32, device="cuda")
        lap_cv_targets(self.h, reps, seed, t)
        return t

    def cv_potentials(self, y, want_phi1=True, want_phi2=True):
        torch = self._torch
        phi1 = torch.empty(self.n, dtype=torch.float64, device="cuda") if want_phi1 else None
        phi2 = torch.empty(self.n, dtype=torch.float64, device="cuda") if want_phi2 else None
        lap_cv_potentials(self.h, y, phi1, phi2)
        return phi1, phi2

    def cv_fit_betas(self, phi1, phi2, seed, first_id, pilot, batches):
        return lap_cv_fit_betas(self.h, phi1, phi2, seed, first_id, pilot, batches)

    def cv_sums(self):
        return lap_cv_sums(self.h, self.n)

    def cv_set_sums(self, a1, a2, p2):
        lap_cv_set_sums(self.h, a1, a2, p2)

    def cv_estimates(self, beta1, beta2, ecc_out=None):
        return lap_cv_estimates(self.h, self.n, beta1, beta2, ecc_out)

    def sample_trace_cv(self, n_samples, seed):
        t = self._torch
        y1 = t.zeros(n_samples, dtype=t.int64, device="cuda")
        y2 = t.zeros(n_samples, dtype=t.int64, device="cuda")
        m2 = t.zeros(n_samples, dtype=t.float64, device="cuda")
        lap_sample_trace_cv(self.h, n_samples, seed, y1, y2, m2)
        return y1, y2, m2


class LapBatch:
    """Many graphs sampled in one persistent CUDA-graph launch (include/lap_batch.h).

    graphs: sequence of (row_ptr, col) host int32 arrays; roots: per-graph
    roots or None (highest degree).  workspace_bytes: device memory lent to
    the sampler (default: 60% of the free device memory, capped at what the
    resident lanes can use).
    """

    def __init__(self, graphs, roots=None, workspace_bytes=None, stream=None):
        import torch
        self._torch = torch
        self.h = lap_batch_create(graphs, roots)
        self.n_graphs = len(graphs)
        s = stream if stream is not None else torch.cuda.current_stream()
        lap_batch_set_stream(self.h, s.cuda_stream)
        info = [lap_batch_graph_info(self.h, g) for g in range(self.n_graphs)]
        self.n = np.array([x[0] for x in info], dtype=np.int64)
        self.arcs = np.array([x[1] for x in info], dtype=np.int64)
        self.roots = np.array([x[2] for x in info], dtype=np.int64)
        self.offsets = np.array([x[3] for x in info] + [int(self.n.sum())], dtype=np.int64)
        self.total_n = int(self.n.sum())
        per_lane = lap_batch_workspace_query(self.h, 1)
        if workspace_bytes is None:
            free, _ = torch.cuda.mem_get_info()
            sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
            workspace_bytes = min(int(free * 0.6), per_lane * sms * 1024)
        workspace_bytes = max(per_lane, (int(workspace_bytes) // per_lane) * per_lane)
        self.workspace = torch.empty(workspace_bytes + 256, dtype=torch.uint8, device="cuda")
        aligned = (self.workspace.data_ptr() + 255) // 256 * 256
        lap_batch_set_workspace(self.h, aligned, workspace_bytes)

    def close(self):
        if self.h is not None:
            lap_batch_destroy(self.h)
            self.h = None
            self.workspace = None
            self._torch.cuda.empty_cache()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, option, value):
        lap_batch_set_option(self.h, option, value)

    def stat(self, which):
        return lap_batch_stat(self.h, which)

    def autotune(self, samples_per_graph, seed, window_ms=300.0):
        return lap_batch_autotune(self.h, samples_per_graph, seed, window_ms)

    def run(self, samples_per_graph, seed):
        lap_batch_run(self.h, samples_per_graph, seed)

    def sync(self):
        lap_batch_sync(self.h)

    def split(self, flat):
        return [flat[self.offsets[g]:self.offsets[g + 1]] for g in range(self.n_graphs)]

    def ecc(self, out=None):
        return lap_batch_ecc(self.h, self.total_n, out)

    def ldiag(self, out=None):
        return lap_batch_ldiag(self.h, self.total_n, out)

    def kemeny(self):
        return lap_batch_kemeny(self.h, self.n_graphs)

    def completion(self):
        return lap_batch_completion(self.h, self.n_graphs)

    def kirchhoff(self):
        return lap_batch_kirchhoff(self.h, self.n_graphs)

    def counts(self, graph, per_node=True):
        return lap_batch_counts(self.h, graph, int(self.n[graph]), per_node)

    def set_path_start(self, graph, start):
        lap_batch_set_path_start(self.h, graph, start)

    def lv_row(self, graph, out=None):
        return lap_batch_lv_row(self.h, graph, int(self.n[graph]), out)

    def mean_wilson_steps(self):
        """Per graph: sum Y1 / omega, the estimate of Tr((I - P_v)^{-1}), the
        expected cost of one Wilson run rooted at the graph's root (Section 3.4)."""
        out = np.zeros(self.n_graphs)
        for g in range(self.n_graphs):
            _, _, s = self.counts(g, per_node=False)
            out[g] = float(s[1]) / float(s[0])
        return out
