/*
 * lap.h - C ABI of the GB300 library for Monte Carlo estimation of Laplacian
 * pseudo-inverse quantities by loop-erased-walk sampling (Liao et al.,
 * "Scalable Algorithms for Laplacian Pseudo-inverse Computation",
 * arXiv 2311.10290).
 *
 * Problem statement (Section 2): G = (V, E) unweighted, undirected and
 * connected, n = |V|, m = |E|, L = D - A, P = D^{-1} A.  A landmark (root) v is
 * fixed (Section 6, "Parameters": the highest-degree node by default).  For
 * every sample id i the library runs, on the GPU,
 *   - one Wilson LE_v run (Section 3.4; Alg. 2 and Alg. 4), counting every
 *     pass of every node (visits) and the total number of walk steps Y1_i,
 *   - one v-absorbed walk from a uniformly drawn start (Alg. 2), counting the
 *     passes of every node,
 *   - one v-absorbed walk from a start drawn from pi(u) = d_u / 2m (Alg. 4),
 *     whose length is Y2_i,
 * and maps the integer counts to (L^+)_uu, electrical closeness centrality
 * c(u) = (n-1) / (n (L^+)_uu + Tr L^+) (Section 2) and Kemeny's constant
 * kappa = E[Y1 - Y2] (Section 5, Alg. 4).
 *
 * Randomness is counter-based (Philox4x32-10, SC'11), keyed by the seed, the
 * sample id, and (node, draw index) for Wilson draws or the step index for the
 * absorbed walks.  Counts are therefore a pure function of (graph, root, seed,
 * sample ids): they do not depend on launch shape, concurrency or how the
 * sample ids are split across calls.
 *
 * Conventions shared by every function:
 *   - Every function returns lap_status; nothing else crosses the ABI.
 *   - Node ids are 0..n-1 in the caller's order.  CSR arrays are int32:
 *     row_ptr[n+1], col_idx[2m]; every edge appears in both rows; rows sorted
 *     strictly ascending (no duplicates); no self-loops; 2m < 2^31.
 *   - A lap_graph handle owns the device memory it allocates; the caller owns
 *     every buffer it passes in.  Handles are not thread-safe.
 *   - Work is queued on the handle's stream (lap_set_stream; default: the
 *     legacy default stream).  lap_sample is asynchronous; functions that
 *     return results synchronise the stream first.
 *   - After an error, lap_last_error(handle) gives a one-line explanation.
 *     Device-side failures (step budget exceeded, CUDA errors) are sticky:
 *     every later call on the handle returns the same status until
 *     lap_set_root resets the handle.
 */
#ifndef LAP_H_
#define LAP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lap_graph lap_graph;

typedef enum {
    LAP_OK = 0,
    LAP_ERR_INVALID_ARG = 1,   /* a NULL pointer, n < 2, a bad option, a seed change, ... */
    LAP_ERR_BAD_CSR = 2,       /* row_ptr not monotone, col out of range, unsorted or duplicate entries */
    LAP_ERR_NOT_SYMMETRIC = 3, /* some arc (u,w) has no reverse arc (w,u) */
    LAP_ERR_SELF_LOOP = 4,
    LAP_ERR_DISCONNECTED = 5,  /* the root does not reach every node (Section 2 assumes G connected) */
    LAP_ERR_TOO_LARGE = 6,     /* 2m >= 2^31, or more than 2^32 sample ids */
    LAP_ERR_OOM = 7,           /* a device allocation failed or the workspace is too small */
    LAP_ERR_NO_SAMPLES = 8,    /* results requested before any sample was drawn */
    LAP_ERR_STEP_LIMIT = 9,    /* a sample exceeded the per-sample step budget */
    LAP_ERR_CUDA = 10,         /* a CUDA runtime error; see lap_last_error */
    LAP_ERR_NO_ROOT = 11       /* lap_set_root has not been called */
} lap_status;

/* Options for lap_set_option. */
typedef enum {
    LAP_OPT_STEP_LIMIT = 1,    /* per-sample budget on each of the three walks' steps; 0 = default
                                  (2^20 + 1024 n); the value is clamped to [1, 2^62] */
    LAP_OPT_SLOTS = 2,         /* samples kept in flight per launch; 0 = as many as the workspace holds */
    LAP_OPT_BLOCK = 3,         /* threads per block of the sampler launch; 0 = automatic */
    LAP_OPT_CURSOR = 4,        /* first sample id of the next lap_sample (default 0); only before the
                                  first sample after lap_set_root.  Lets several processes or GPUs
                                  draw disjoint sample-id ranges whose counts add up exactly. */
    LAP_OPT_KERNEL = 5,        /* 0 = automatic: kernel 3 for calls of at most 320 samples per SM
                                  (1024 when the graph's arrays exceed 96 MB) on graphs of at
                                  least 2^14 nodes when it applies, else kernel 2 when n < 2^27,
                                  else kernel 1.
                                  1 = 8-byte state per node.
                                  2 = 1-byte state per node.  Kernel 2 keeps draw counts above 30
                                  (and, with LAP_OPT_PATHS = 1, path departure counts above 14) in
                                  a table per sample of 8-byte entries, as many as the next power
                                  of two >= n, 256 to 8192.  A sample that does not fit kernel 2
                                  (more such nodes than the table holds, or a loop-erased path
                                  longer than the stack) is withdrawn and re-run with kernel 1.
                                  3 = several walkers per sample (LAP_OPT_WALKERS lanes share one
                                  Wilson run; 2 bytes of state per node): more independent memory
                                  chains when a call has few samples, and each sample finishes
                                  sooner.  Kernel 3 needs n < 2^22 and covers every estimator
                                  form (LAP_OPT_PATHS 0 or 1, with or without the control
                                  variate; 2 more bytes per node with LAP_OPT_PATHS = 1).  Its
                                  samples that do not fit (a node drawn 1023 times, a path longer
                                  than a walker's stack, a walker without progress for 4 s, a node
                                  left 255 times by one loop-included path) are withdrawn and
                                  re-run with kernel 1.
                                  Counts are identical with every kernel. */
    LAP_OPT_STACK = 6,         /* loop-erased path capacity per sample (kernel 2) or walker (kernel 3); 0 = default
                                  (16 sqrt(n) rounded up to a power of two, at least 1024) */
    LAP_OPT_PATHS = 7,         /* 0 (default): the uniform-start and pi-start v-absorbed walks take
                                  their own draws, as Alg. 2 and Alg. 4 print them.  1: they are the
                                  loop-included paths of the sample's own Wilson stacks (Section 4.2,
                                  "loop-erased walk" lemma and "Sample from the paths"; Section 5.2):
                                  same starts, and the j-th departure of a path from u takes u's
                                  stack entry j, the draw (u, j, i, 0) of the Wilson run.  Same
                                  expectations (so the same estimands), correlated with the Wilson
                                  counts, which lowers the variance of y1 - 2 y2 and of Y1 - Y2.
                                  Only before the first sample after lap_set_root. */
    LAP_OPT_WALKERS = 9,       /* lanes per sample of kernel 3: 2, 4, 8 or 16; 0 (default) = 16 when
                                  the call's samples times 16 lanes fit on the GPU at once (1280
                                  lanes per SM), else 8.  The path stacks of a sample hold 8 x
                                  LAP_OPT_STACK entries in all, shared out among its walkers;
                                  with 16 walkers a node drawn 511 times withdraws the sample.  They run the
                                  sample's Wilson run together (Section 3.4, stack representation:
                                  the popped cycles, so every node's draws and the tree, do not
                                  depend on the order in which walkers find them), then one runs
                                  the uniform-start walk and one the pi-start walk. */
    LAP_OPT_PATH_START = 8     /* -1 (default): the first absorbed walk (or loop-included path) of
                                  each sample starts at a uniform draw (Alg. 2).  s in [0, n): it
                                  starts at node s, so its passes of u have mean d_u (L_v^{-1})_{su}
                                  (Section 4.2, "v-absorbed walk" and "loop-erased walk" lemmas)
                                  and lap_lv_row returns row s of L_v^{-1}; with root t,
                                  (L_t^{-1})_{ss} is the effective resistance between s and t.  The
                                  ECC outputs (lap_ecc, lap_ldiag, lap_kirchhoff,
                                  lap_rw_betweenness, the CV ECC) are then refused
                                  (LAP_ERR_INVALID_ARG); Wilson counts and lap_kemeny are unchanged.
                                  Only before the first sample after lap_set_root. */
} lap_option;

/* Statistics for lap_get_stat. */
typedef enum {
    LAP_STAT_SLOTS = 1,        /* samples in flight per launch of a large call (LAP_STAT_KERNEL) with
                                  the current workspace (kernel 3: groups of walkers) */
    LAP_STAT_KERNEL = 2,       /* kernel a large lap_sample call will use (1, 2 or 3) */
    LAP_STAT_FALLBACKS = 3,    /* samples re-run with kernel 1 after kernel 2 or 3 withdrew them, since
                                  lap_set_root (synchronises) */
    LAP_STAT_LAST_KERNEL = 4   /* kernel of the last lap_sample call (0 before any) */
} lap_stat;

/* Library version as major*10000 + minor*100 + patch. */
int32_t lap_version(void);

/*
 * Ingest a CSR graph (row a1 of the hot path: the graph model of Section 2).
 *   n              number of nodes, >= 2.
 *   row_ptr        int32[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = 2m.
 *   col_idx        int32[2m].
 *   ptrs_on_device 0: both pointers are host memory; 1: both are device memory
 *                  (e.g. torch CUDA tensors) on the current device.
 *   out            receives the new handle; *out is NULL on failure.
 * The arrays are copied; the caller keeps ownership of its buffers.  The CSR
 * is validated on the GPU (monotone row_ptr, col range, strictly ascending
 * rows, no self-loop, symmetry) and degrees and per-node row records are
 * built.  Errors: LAP_ERR_INVALID_ARG, LAP_ERR_BAD_CSR, LAP_ERR_SELF_LOOP,
 * LAP_ERR_NOT_SYMMETRIC, LAP_ERR_TOO_LARGE, LAP_ERR_OOM, LAP_ERR_CUDA.  On error
 * nothing is allocated and the reason is available from lap_last_error(NULL).
 */
lap_status lap_graph_create(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                            int ptrs_on_device, lap_graph **out);

/* Frees all device memory the handle owns.  Accepts NULL. */
lap_status lap_graph_destroy(lap_graph *g);

/* Queue all later work of the handle on `cuda_stream` (a cudaStream_t, e.g.
 * torch.cuda.current_stream().cuda_stream); NULL selects the legacy default
 * stream. */
lap_status lap_set_stream(lap_graph *g, void *cuda_stream);

/* Set an option (see lap_option). */
lap_status lap_set_option(lap_graph *g, int32_t option, int64_t value);

/*
 * Device workspace for the per-sample Wilson state (8 bytes per node per
 * sample in flight with kernel 1; with kernel 2, n rounded up to 256 (twice
 * that with LAP_OPT_PATHS = 1), plus 4 bytes per stack entry, plus the count
 * table (8 bytes times the next power of two >= n, 2 KB to 64 KB), rounded up
 * to 256).  lap_workspace_query returns the bytes the
 * current kernel needs to keep `slots` samples in flight.  lap_set_workspace lends the handle a caller-owned
 * device buffer (at least 8*n bytes, 256-byte aligned), which must stay alive
 * while the handle uses it; the handle zeroes it.  Without a workspace,
 * lap_sample allocates one itself (up to 1/2 of the free device memory).
 */
lap_status lap_workspace_query(const lap_graph *g, uint64_t slots, uint64_t *bytes);
lap_status lap_set_workspace(lap_graph *g, void *device_ptr, uint64_t bytes);

/*
 * Choose the landmark v (Section 3.1: L^+ does not depend on v, so an
 * easy-to-hit node is picked; Section 6: the highest-degree node).
 *   v >= 0  use node v;   v < 0  the highest-degree node, smallest id on ties.
 * A breadth-first search from v on the GPU checks that v reaches all n nodes
 * (LAP_ERR_DISCONNECTED otherwise) and records hop distances.  Resets all
 * counts, the sample cursor and the seed, and clears a sticky error.
 * root_out (may be NULL) receives the chosen v.
 */
lap_status lap_set_root(lap_graph *g, int32_t v, int32_t *root_out);

/*
 * Draw sample ids [cursor, cursor + n_samples) and add their counts (the
 * cursor starts at 0, or at LAP_OPT_CURSOR)
 * (Alg. 2 and Alg. 4; hot-path rows a2-a5).  Asynchronous.  The first call
 * after lap_set_root fixes the seed; a later call with another seed returns
 * LAP_ERR_INVALID_ARG.  Two calls of k/2 samples give exactly the counts of
 * one call of k.  Errors: LAP_ERR_NO_ROOT, LAP_ERR_INVALID_ARG,
 * LAP_ERR_TOO_LARGE (cursor would pass 2^32), LAP_ERR_OOM, LAP_ERR_CUDA; a step
 * budget overrun is reported as LAP_ERR_STEP_LIMIT by the next synchronising
 * call.
 */
lap_status lap_sample(lap_graph *g, uint64_t n_samples, uint64_t seed);

/*
 * lap_sample that also writes each sample's Y1 (Wilson steps, loops
 * included) and Y2 (pi-start walk length) to device arrays y1_dev[n_samples],
 * y2_dev[n_samples] (caller-owned device memory; entry q belongs to sample id
 * cursor + q).  Both pointers must be set, or both NULL (then it is
 * lap_sample).  Used for variance estimates and sampled parity checks.
 */
lap_status lap_sample_trace(lap_graph *g, uint64_t n_samples, uint64_t seed, uint64_t *y1_dev, uint64_t *y2_dev);

/* Wait for queued work and report a device-side failure, if any. */
lap_status lap_sync(lap_graph *g);

/*
 * Results (hot-path row a6, FP64).  With omega samples drawn:
 *   y1(u) = cnt1[u]/(omega d_u) ~ (L_v^{-1})_uu,
 *   y2(u) = cnt2[u]/(omega d_u) ~ (1/n) e_u^T L_v^{-1} 1,
 *   (L^+)_uu = y1(u) - 2 y2(u) + (1/n) sum_w y2(w)   (u != v),
 *   (L^+)_vv = (1/n) sum_w y2(w)                      (Section 3.1, element-wise Thm 1),
 *   c(u) = (n-1) / (n (L^+)_uu + sum_w (L^+)_ww)      (Section 2),
 *   kappa = (sum_i Y1_i - sum_i Y2_i) / omega         (Alg. 4).
 * For very small omega the estimated denominator of c(u) can be <= 0; the
 * raw IEEE result is returned.  `out` has n doubles (1 for lap_kemeny); it is
 * host memory when out_on_device = 0, device memory otherwise.  These calls
 * synchronise the handle's stream.  Errors: LAP_ERR_NO_ROOT,
 * LAP_ERR_NO_SAMPLES, LAP_ERR_INVALID_ARG, sticky errors.
 */
lap_status lap_ecc(lap_graph *g, double *out, int out_on_device);
lap_status lap_ldiag(lap_graph *g, double *out, int out_on_device);
lap_status lap_kemeny(lap_graph *g, double *out1);

/*
 * Passes of the first absorbed walk per node, scaled: out[u] = cnt2[u] /
 * (omega d_u) (n doubles, host or device memory by out_on_device).  With a
 * fixed start s (LAP_OPT_PATH_START) this estimates row s of L_v^{-1},
 * (L_v^{-1})_{su} (Section 4.2, "v-absorbed walk" lemma: the walk from s
 * passes u d_u (L_v^{-1})_{su} times on average; the same for the
 * loop-included path, "loop-erased walk" lemma); out[v] = 0.  With the uniform
 * start it is y2(u) ~ (1/n) e_u^T L_v^{-1} 1 of Alg. 2.  Synchronises.
 * Errors: LAP_ERR_NO_ROOT, LAP_ERR_NO_SAMPLES, LAP_ERR_INVALID_ARG, sticky
 * errors.
 */
lap_status lap_lv_row(lap_graph *g, double *out, int out_on_device);

/*
 * Solves L_v x = b in FP64 (L_v: the Laplacian without row and column v,
 * Section 3.1; symmetric positive definite for a connected graph) by
 * conjugate gradients with the Jacobi preconditioner D^{-1}, until
 * ||b - L_v x|| <= rtol ||b|| or maxiter iterations.  b[v] is ignored and
 * x[v] = 0.  The sampled quantities that are linear in L_v^{-1} applied to a
 * known vector come out exactly: b = 1 gives n y2(u) of Alg. 2 and the
 * row-sum terms of (L^+)_uu (Section 3.1, element-wise Theorem 1); b = d
 * gives the hitting times h(u, v) and E[Y2] = d^T x / 2m (Section 3.2,
 * Alg. 4); b = e_s gives row s of L_v^{-1}.  b, x: n doubles, host or
 * device (on_device); iterations and residual (may be NULL) receive the
 * iterations run and the final relative residual.  Synchronises; allocates
 * and frees 4 n + 2056 doubles of device scratch.  Errors: LAP_ERR_NO_ROOT,
 * LAP_ERR_INVALID_ARG, LAP_ERR_OOM, LAP_ERR_CUDA.
 */
lap_status lap_lv_solve(lap_graph *g, const double *b, double *x, int on_device, double rtol, int32_t maxiter,
                        int32_t *iterations, double *residual);

/*
 * Two more quantities of the same diagonal (Section 5, "Discussions"):
 *   lap_kirchhoff       the Kirchhoff index as the paper defines it,
 *                       Tr(L^+) = sum_u (L^+)_uu (the sum of resistances
 *                       over node pairs is n times this); out1: one double;
 *   lap_rw_betweenness  random-walk betweenness for every node,
 *                       c_b(u) = 1/n + Tr(L^+) / ((n-1) (Tr(L^+) + n (L^+)_uu));
 *                       out: n doubles, host or device (out_on_device).
 * Computed from the same estimates as lap_ecc (same samples, same sums).
 * Synchronise.  Errors as lap_ecc.
 */
lap_status lap_kirchhoff(lap_graph *g, double *out1);
lap_status lap_rw_betweenness(lap_graph *g, double *out, int out_on_device);

/*
 * SpanTree estimators (Alg. 1 for ECC, Alg. 3 for Kemeny's constant;
 * Section 4.1 and Section 5.1), on the same handle and root, with their own
 * sample ids (0, 1, ... since lap_set_root) and sums:
 *   lap_spantree_sample     draws n_samples uniform spanning trees rooted at v
 *                           (Wilson's algorithm with the Philox keying of
 *                           lap_sample, so tree i equals the tree of
 *                           lap_sample's sample id i) and adds, for every node u,
 *                           the integer flow sums along u's BFS path (the BFS
 *                           parent of u is its smallest-id neighbour one hop
 *                           closer to v):
 *                             x1(u)   unit current u -> v on the tree,
 *                             x2(u)   1/n injected at every node (times n),
 *                             x2d(u)  d_w/2m injected at every w (times 2m).
 *                           Synchronises.  Uses the handle's workspace (8 n bytes
 *                           per tree in flight) and allocates per-CTA scratch.
 *   lap_spantree_sums       the integer sums (int64[n] each, any may be NULL) and
 *                           the number of trees; host or device (on_device).
 *   lap_spantree_estimates  (L^+)_uu = x1/omega - 2 x2/(n omega) + (1/n) sum x2/(n omega),
 *                           ECC as lap_ecc, and
 *                           kappa = sum_u d_u x1(u)/omega - sum_u d_u x2d(u)/(2m omega);
 *                           ldiag/ecc: n doubles (may be NULL), kemeny: one double.
 * The estimators are unbiased with bounded per-sample range (Section 4.1,
 * Hoeffding bound).  Errors: LAP_ERR_NO_ROOT, LAP_ERR_INVALID_ARG (seed change),
 * LAP_ERR_NO_SAMPLES, LAP_ERR_STEP_LIMIT, LAP_ERR_OOM, sticky errors.
 */
lap_status lap_spantree_sample(lap_graph *g, uint64_t n_samples, uint64_t seed);
lap_status lap_spantree_sums(lap_graph *g, int64_t *x1, int64_t *x2, int64_t *x2d, uint64_t *omega, int on_device);
lap_status lap_spantree_estimates(lap_graph *g, double *ldiag, double *ecc, int on_device, double *kemeny);

/*
 * Raw integer state (for parity checks and checkpointing):
 *   cnt1[n]  visits per node summed over samples (0 at v),
 *   cnt2[n]  passes of the uniform-start walks per node,
 *   sums[4]  = { omega (samples drawn), sum Y1, sum Y2, seed }.
 * Any pointer may be NULL.  Host memory when on_device = 0.  Synchronises.
 */
lap_status lap_counts(lap_graph *g, uint64_t *cnt1, uint64_t *cnt2, uint64_t *sums, int on_device);

/*
 * Replaces the handle's counts with given totals, in lap_counts' layout:
 * cnt1[n], cnt2[n] and sums[3] = { omega, sum Y1, sum Y2 }.  The use is the
 * one exchange step of a run split over processes or GPUs: each draws a
 * disjoint sample-id range (LAP_OPT_CURSOR), the integer counts are summed
 * (an all-reduce of 16 n + 24 bytes), and one handle finalizes the totals
 * with lap_ecc / lap_ldiag / lap_kemeny, exactly as if it had drawn every
 * sample itself (Alg. 2 and Alg. 4 estimate from these sums only).  Also
 * restores a checkpoint taken with lap_counts.  Requires lap_set_root (same
 * root as the counts); cnt1[v] must be 0 and cnt1[u] >= omega >= 1 for
 * u != v (else LAP_ERR_INVALID_ARG).  Control-variate sums are not part of
 * the state and are cleared.  Later lap_sample calls add to these totals
 * (ids continue from the handle's cursor).  Host or device buffers
 * (on_device).  Synchronises.
 */
lap_status lap_set_counts(lap_graph *g, const uint64_t *cnt1, const uint64_t *cnt2, const uint64_t *sums, int on_device);

/* ------------------------------------------------------------------------
 * Learned control variate.  The paper has no control variate; these entry
 * points add one that keeps every estimator unbiased.  For an integer
 * potential h on nodes and S[u] = sum of h over N(u), each random step
 * u -> w contributes d_u h[w] - S[u], which has mean exactly zero given u.
 *   Wilson draws (potential h1):  Z1[u] = d_u A1[u] - cnt1[u] S1[u],
 *       A1[u] = sum of h1[w] over the draws at u;
 *       ECC uses y1_cv(u) = (cnt1[u] - beta1 Z1[u] / d_u) / (omega d_u).
 *   pi-start walks (potential h2): M2 = sum_u (d_u A2[u] - P2[u] S2[u]) / d_u,
 *       A2[u] = sum of h2[w] over the pi-walk steps at u, P2[u] = their number;
 *       Kemeny uses kappa_cv = (sum Y1 - sum Y2 + beta2 M2) / omega.
 * With h2 = the hitting time h(., v) (Section 3.2, v-absorbed walks), Y2 - M2
 * equals the hitting time of the walk's start: the walk's own randomness
 * cancels.  Potentials come from the MLP (8 -> 64 -> 64 -> 2) over the node
 * features below; beta1, beta2 must be chosen independently of the samples
 * they are applied to (e.g. from a pilot run) for unbiasedness.
 * ------------------------------------------------------------------------ */

/* Packed FP32 MLP parameters: W1[64][8] b1[64] W2[64][64] b2[64] W3[2][64] b3[2]. */
#define LAP_MLP_PARAMS 4866

/* 8 features per node into feat_dev[n][8] (device, float):
 * ln d_u, 1/d_u, ln(1 + hop distance to v), [u adjacent to v], ln(mean
 * neighbour degree), share of degree-1 neighbours, ln(two-hop degree sum /
 * one-hop degree sum), P(walk from u hits v within 8 steps).  Needs the root. */
lap_status lap_features(lap_graph *g, float *feat_dev);

/* Hitting-time targets: for every node u, `reps` v-absorbed walks from u
 * (step t of repetition r uses Philox counter (t, u, r, 3)); sums_dev[n]
 * (device uint64) is overwritten with the total lengths, so sums/reps
 * estimates h(u, v) = (L_v^{-1} d)_u.  Synchronises. */
lap_status lap_hitting_walks(lap_graph *g, uint32_t reps, uint64_t seed, uint64_t *sums_dev);

/*
 * Training targets of the control variate's network for one graph (device
 * float[n][2]), from the samples drawn since lap_set_root and `reps`
 * v-absorbed walks from every node (lap_hitting_walks with `seed`):
 *   targets[u][0] = cnt1[u] / omega            (mean Wilson visits, d_u (L_v^{-1})_uu;
 *                                               LE-walk lemma of Section 3.4)
 *   targets[u][1] = (walk sum[u] / reps) / Ybar2 (hitting time h(u, v), Section 3.2,
 *                                               over Ybar2 = max(sum Y2 / omega, 1e-9),
 *                                               the estimate of E[Y2] = sum_u pi(u) h(u, v))
 * Both are computed in FP64 and rounded to float; row v is zero (leave it
 * out of training).  Synchronises.  Errors: LAP_ERR_NO_ROOT,
 * LAP_ERR_NO_SAMPLES, LAP_ERR_INVALID_ARG, LAP_ERR_STEP_LIMIT, LAP_ERR_OOM.
 */
lap_status lap_cv_targets(lap_graph *g, uint32_t reps, uint64_t seed, float *targets_dev);

/*
 * Potentials from the network's outputs y_dev[n][2] (device float, as
 * lap_mlp_forward writes them for the node features):
 *   phi1[u] = y[u][0] / d_u                 (~ (L_v^{-1})_uu),
 *   phi2[u] = y[u][1] * (sum Y2 / omega)    (~ h(u, v)), phi2[v] = 0,
 * the scale being the mean pi-walk length of the samples drawn since
 * lap_set_root (draw a few pilot samples first, e.g. at LAP_OPT_CURSOR ids
 * kept apart from the estimate's).  Device double[n] outputs, either may be
 * NULL (phi2 then needs no samples).  Synchronises.
 */
lap_status lap_cv_potentials(lap_graph *g, const float *y_dev, double *phi1_dev, double *phi2_dev);

/*
 * Coefficients of the two control variates from pilot samples, so that they
 * do not depend on the samples of the estimate (which keeps it unbiased):
 * sets the potentials (as lap_cv_set_potentials; either may be NULL), draws
 * `batches` batches of pilot / batches samples with ids from first_id on,
 * then
 *   beta1 = sum_u sum_b (V_bu - Vbar_u)(Z_bu - Zbar_u) / sum_u sum_b (Z_bu - Zbar_u)^2,
 *           V_bu = visits of u in batch b, Z_bu = Z1_b(u) / d_u (least squares
 *           of the ECC variate, pooled over nodes; 0 without phi1),
 *   beta2 = -cov(Y1 - Y2, M2) / var(M2) over the pilot samples (least
 *           squares of the Kemeny variate; 0 without phi2),
 * and resets the handle as lap_set_root does (counts and cursor cleared, the
 * potentials kept).  Needs lap_set_root and no sample drawn since;
 * 2 <= batches <= 64, 1 <= pilot / batches <= 2^24, ids below 2^32.
 * Synchronises; allocates and frees temporary device buffers (16 n batches +
 * 24 pilot bytes).  Errors: LAP_ERR_NO_ROOT, LAP_ERR_INVALID_ARG,
 * LAP_ERR_TOO_LARGE, LAP_ERR_OOM, LAP_ERR_STEP_LIMIT, LAP_ERR_CUDA.
 */
lap_status lap_cv_fit_betas(lap_graph *g, const double *phi1_dev, const double *phi2_dev, uint64_t seed,
                            uint64_t first_id, uint64_t pilot, uint32_t batches, double *beta1, double *beta2);

/* Potentials phi1 (Wilson draws, ECC) and phi2 (pi walks, Kemeny) as device
 * double[n]; either may be NULL (that term off).  They are quantised to
 * h = round(2^16 phi).  Only before the first sample after lap_set_root;
 * lap_set_root clears the sums and keeps the potentials. */
lap_status lap_cv_set_potentials(lap_graph *g, const double *phi1_dev, const double *phi2_dev);

/* Raw control-variate sums a1[n], a2[n], p2[n] (int64; NULL skips). */
lap_status lap_cv_sums(lap_graph *g, int64_t *a1, int64_t *a2, int64_t *p2, int on_device);

/* Replaces the control-variate sums a1[n], a2[n], p2[n] (int64, lap_cv_sums'
 * layout; host or device) with given totals, for example the sums of
 * several handles or processes that drew disjoint sample ids with the same
 * potentials (call after lap_set_counts, which clears them).  Needs the
 * potentials set.  Synchronises. */
lap_status lap_cv_set_sums(lap_graph *g, const int64_t *a1, const int64_t *a2, const int64_t *p2, int on_device);

/* Control-variate estimates: ldiag[n], ecc[n] (either may be NULL), kemeny[1]
 * and m2_total[1] (host doubles; may be NULL).  Synchronises. */
lap_status lap_cv_estimates(lap_graph *g, double beta1, double beta2, double *ldiag, double *ecc, int on_device,
                            double *kemeny, double *m2_total);

/* lap_sample_trace that also writes each sample's M2 to m2_dev[n_samples]
 * (device double).  Needs phi2 set. */
lap_status lap_sample_trace_cv(lap_graph *g, uint64_t n_samples, uint64_t seed, uint64_t *y1_dev, uint64_t *y2_dev,
                               double *m2_dev);

/* MLP kernels.  LAP_MLP_TCGEN05 (the default): fifth-generation tensor-core
 * products (tcgen05.mma, operands in shared memory, FP32 accumulators in
 * tensor memory), 128 rows per tile; a product that does not complete within
 * 1 s makes the call write NaN to its outputs (forward) or its loss
 * (training).  LAP_MLP_MMA_SYNC: the warp-level mma.sync.m16n8k16 kernel,
 * kept for comparison.  Both round at the same points (BF16 operands, FP32
 * accumulation, FP32 bias gradients); they differ only in FP32 summation
 * order.  lap_mlp_select sets the kernel for every later MLP call of the
 * process (not per stream); LAP_ERR_INVALID_ARG for any other value. */
enum lap_mlp_kernel { LAP_MLP_TCGEN05 = 0, LAP_MLP_MMA_SYNC = 1 };
lap_status lap_mlp_select(int32_t kernel);

/* MLP forward on rows x[rows][8] -> y[rows][2] (device float), BF16 tensor
 * cores with FP32 accumulation; params: LAP_MLP_PARAMS device floats. */
lap_status lap_mlp_forward(const float *params_dev, const float *x_dev, int64_t rows, float *y_dev, void *cuda_stream);

/* MSE loss (1/rows) sum_i (w0 (y_i0 - t_i0)^2 + w1 (y_i1 - t_i1)^2) and its
 * gradient w.r.t. the packed parameters; grad_dev[LAP_MLP_PARAMS] and
 * loss_dev[1] (device float) are overwritten. */
lap_status lap_mlp_loss_grad(const float *params_dev, const float *x_dev, const float *t_dev, int64_t rows, float w0,
                             float w1, float *grad_dev, float *loss_dev, void *cuda_stream);

/* One AdamW step (decoupled weight decay) on count FP32 parameters in place;
 * m_dev, v_dev are the moment buffers (zero before step 1); step >= 1. */
lap_status lap_adamw(float *params_dev, float *m_dev, float *v_dev, const float *grad_dev, int64_t count, int32_t step,
                     float lr, float beta1, float beta2, float eps, float weight_decay, void *cuda_stream);

/* Read a statistic (see lap_stat) into *value. */
lap_status lap_get_stat(lap_graph *g, int32_t stat, int64_t *value);

/* Hop distance from the root for every node (int32[n]; host when
 * on_device = 0), as found by the connectivity check of lap_set_root. */
lap_status lap_hops(lap_graph *g, int32_t *out, int on_device);

/* Number of nodes, arcs (2m) and the current root (-1 when unset). */
lap_status lap_graph_info(const lap_graph *g, int32_t *n, int64_t *arcs, int32_t *root);

/*
 * lap_sample_static - the sampler for callers that must not allocate device
 * memory.  The paper has no counterpart: this entry point exists for code that
 * runs where cudaMalloc is unavailable or forbidden, such as a plug-in whose
 * host application owns all device memory through its own pool, a real-time
 * service that must keep a fixed memory footprint after start-up, or a thread
 * that must not trigger the device-wide synchronisation cudaMalloc/cudaFree can
 * cause.  It computes exactly what lap_graph_create + lap_set_root +
 * lap_sample + lap_counts compute for the same graph, root, seed and sample ids,
 * but takes the graph and the outputs as caller-owned device buffers and keeps
 * all of its scratch (row records, counters, per-sample Wilson state) in one
 * fixed array of lap_static_scratch_bytes() = 32 MiB that the library holds
 * on every GPU that loads it, until the process exits.  It never calls
 * cudaMalloc, cudaFree or any allocating library routine.
 *
 *   n, row_ptr, col_idx  CSR as for lap_graph_create, in DEVICE memory
 *                        (not validated here: pass a valid, connected graph)
 *   root                 landmark v, or < 0 for the highest-degree node
 *   seed, first_id       Philox seed and first sample id; ids
 *                        [first_id, first_id + n_samples) are drawn and
 *                        must lie below 2^32 (else LAP_ERR_TOO_LARGE)
 *   cnt1, cnt2           device uint64[n], overwritten with the visit and
 *                        uniform-walk pass counts (as lap_counts)
 *   sums2                device uint64[2], overwritten with {sum Y1, sum Y2}
 *   cuda_stream          stream to run on (NULL: legacy default stream)
 *
 * The graph must fit the scratch with at least one sample in flight
 * (24 n + 512 bytes, so n up to about 1.39 million): larger graphs return
 * LAP_ERR_TOO_LARGE.  Smaller graphs keep up to (32 MiB - 16 n) / (8 n)
 * samples in flight.  The call synchronises the stream before returning: it
 * reads row_ptr[n] (and, for root < 0, the chosen root) back to the host, and
 * the device status after the samples.  The first call on a device (and the
 * first after that device's context was re-created, e.g. by cudaDeviceReset)
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share
 * the one array, which keeps the last call's contents; each call clears what
 * must start at zero, so calls that overlap on the GPU (other streams or
 * threads) race and give wrong results: serialise them.
 * Errors (LAP_ERR_INVALID_ARG, LAP_ERR_TOO_LARGE, LAP_ERR_STEP_LIMIT for a
 * sample over the step budget or a node drawn from more than 2^30 times in
 * one sample, LAP_ERR_CUDA) are explained by lap_static_last_error().
 * Argument and size errors are found on the host before any CUDA call.
 */
lap_status lap_sample_static(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t root,
                             uint64_t seed, uint64_t first_id, uint64_t n_samples,
                             uint64_t *cnt1, uint64_t *cnt2, uint64_t *sums2, void *cuda_stream);

/* Size in bytes of the fixed scratch array used by lap_sample_static. */
uint64_t lap_static_scratch_bytes(void);

/* One-line description of the last lap_sample_static error of this thread. */
const char *lap_static_last_error(void);

/* One-line description of the last error on this handle (or of the last
 * failed lap_graph_create when g is NULL).  Never NULL. */
const char *lap_last_error(const lap_graph *g);

#ifdef __cplusplus
}
#endif

#endif /* LAP_H_ */
