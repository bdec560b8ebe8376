/*
 * lap_batch.h - batches of graphs sampled in one persistent launch.
 *
 * Many independent problems of the kind lap.h solves (each an unweighted,
 * undirected, connected graph with its own landmark v; Section 2, Section 6
 * "Parameters") are sampled together: every graph gets the same number of
 * samples omega, and graph g's sample ids 0 .. omega-1 use the same Philox
 * keying as lap_sample (Alg. 2 Wilson LE_v run and uniform-start walk; Alg. 4
 * pi-start walk).  Graph g's counts, (L^+)_uu, ECC and Kemeny estimate are
 * therefore bit-identical to those of a lap_graph handle on that graph with
 * the same root and seed after lap_sample(omega, seed).
 *
 * One run is one CUDA graph launch on the handle's stream: counter resets,
 * the persistent sampler over a queue of work units {graph, first sample}
 * (up to `claim` consecutive samples of one graph each, largest graphs first
 * by default), and the FP64 finalize of every graph.  Samples whose state
 * does not fit one byte per node are re-run with the 8-byte kernel when the
 * results are first read (lap_batch_stat LAP_BSTAT_RERUNS counts them).
 *
 * Conventions are those of lap.h: every function returns lap_status, the
 * caller owns every buffer it passes, handles are not thread-safe, and
 * lap_batch_last_error explains the last error of a handle.
 */
#ifndef LAP_BATCH_H_
#define LAP_BATCH_H_

#include "lap.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lap_batch lap_batch;

/* Options for lap_batch_set_option. */
typedef enum {
    LAP_BOPT_LANES = 1,  /* samples in flight (one per GPU thread); 0 = as many as the workspace
                            and the resident-thread capacity allow */
    LAP_BOPT_CLAIM = 2,  /* samples per work unit (1 .. 65536); default 1 */
    LAP_BOPT_ORDER = 3,  /* unit order: 0 = largest graphs first (default), 1 = smallest first,
                            2 = the caller's graph order */
    LAP_BOPT_BLOCK = 4,  /* threads per block; 0 = automatic */
    LAP_BOPT_STACK = 5,  /* loop-erased path capacity per lane; 0 = 16 sqrt(largest n), at least 1024 */
    LAP_BOPT_PATHS = 6   /* LAP_OPT_PATHS for every graph of the batch (0 default, 1 loop-included paths) */
} lap_batch_option;

/* Statistics for lap_batch_stat. */
typedef enum {
    LAP_BSTAT_LANES = 1,         /* lanes the next run uses */
    LAP_BSTAT_CLAIM = 2,         /* samples per work unit */
    LAP_BSTAT_UNITS = 3,         /* work units of the last run */
    LAP_BSTAT_RERUNS = 4,        /* samples of the last run re-run with the 8-byte kernel */
    LAP_BSTAT_GRAPH_CAPTURES = 5 /* CUDA graphs captured by this handle so far */
} lap_batch_stat_id;

/*
 * Creates a batch from n_graphs host CSR graphs (layout and validity rules
 * of lap_graph_create): graph g has n[g] >= 2 nodes, row_ptr[g] (n[g]+1
 * entries) and col_idx[g] (row_ptr[g][n[g]] entries).  roots[g] is its
 * landmark v, or < 0 for its highest-degree node (smallest id on ties);
 * roots may be NULL (all < 0).  The graphs are copied to the device (packed
 * arenas), validated and checked for connectivity from their roots; the
 * caller's buffers are not kept.  Graphs passed with the same n and the same
 * row_ptr and col_idx pointers share one device copy of the CSR (one graph
 * sampled from several roots, e.g. a landmark study: Section 6).
 * 1 <= n_graphs <= 65535; the arcs of all graphs together must be fewer than
 * 2^40.
 * Errors: LAP_ERR_INVALID_ARG, LAP_ERR_BAD_CSR, LAP_ERR_NOT_SYMMETRIC,
 * LAP_ERR_SELF_LOOP, LAP_ERR_DISCONNECTED (naming the graph), LAP_ERR_OOM,
 * LAP_ERR_CUDA; explained by lap_batch_last_error(NULL).
 */
lap_status lap_batch_create(int32_t n_graphs, const int32_t *n, const int32_t *const *row_ptr,
                            const int32_t *const *col_idx, const int32_t *roots, lap_batch **out);

lap_status lap_batch_destroy(lap_batch *b);

/* Stream for every later call (NULL: legacy default stream). */
lap_status lap_batch_set_stream(lap_batch *b, void *cuda_stream);

/* Sets a lap_batch_option; value >= 0. */
lap_status lap_batch_set_option(lap_batch *b, int32_t option, int64_t value);

/* Device bytes of the Wilson-state workspace for `lanes` samples in flight
 * (one slot per lane: a state byte per node of the largest graph, rounded up
 * to 256 (twice that with LAP_BOPT_PATHS = 1), plus the path stack and a
 * table of counts above 30: 8 bytes times the next power of two >= that n,
 * 2 KB to 64 KB). */
lap_status lap_batch_workspace_query(const lap_batch *b, uint64_t lanes, uint64_t *bytes);

/* Lends the handle device memory for the workspace (256-byte aligned; the
 * caller keeps ownership and must keep it alive while the handle uses it).
 * Without it, the first run allocates half of the free device memory. */
lap_status lap_batch_set_workspace(lap_batch *b, void *device_ptr, uint64_t bytes);

/*
 * Picks LAP_BOPT_LANES and LAP_BOPT_CLAIM for runs of samples_per_graph
 * samples: each candidate runs the sampler for window_ms milliseconds per
 * lane, starting at three points of the work queue (its start, one third,
 * two thirds), and scores walk steps per second of kernel time.  Candidates:
 * lanes = 1/4, 1/2, 3/4 and all of the maximum with claim 1, then claim 4
 * and 16 at the best lane count.  Writes up to max_trials rows (lanes,
 * claim, steps/s) to the optional arrays and their number to *n_trials.
 * The probes leave no counts behind (every run resets them).
 */
lap_status lap_batch_autotune(lap_batch *b, uint64_t samples_per_graph, uint64_t seed, double window_ms,
                              int32_t max_trials, int64_t *trial_lanes, int32_t *trial_claim,
                              double *trial_steps_per_s, int32_t *n_trials);

/*
 * Draws sample ids 0 .. samples_per_graph-1 of every graph with `seed`
 * (counts of any earlier run are discarded) and finalizes every graph.
 * Asynchronous: one CUDA graph launch on the handle's stream (re-captured
 * when the sample count, seed or a launch option changed).
 * 1 <= samples_per_graph <= 2^31.
 */
lap_status lap_batch_run(lap_batch *b, uint64_t samples_per_graph, uint64_t seed);

/* Synchronises, re-runs withdrawn samples if any, checks device status.
 * Device failures (step budget, CUDA) are sticky until the next run. */
lap_status lap_batch_sync(lap_batch *b);

/* Per-graph results of the last run (synchronise first):
 *   lap_batch_ecc / lap_batch_ldiag   double[total nodes]: graph g's values at
 *                                     node offset lap_batch_graph_info(g).offset,
 *                                     host or device buffer (on_device)
 *   lap_batch_kemeny                  double[n_graphs] (host)
 *   lap_batch_completion              double[n_graphs] (host): seconds from the
 *                                     sampler's start to the end of the graph's
 *                                     last sample (re-runs not included)
 *   lap_batch_counts                  graph g's cnt1, cnt2 (uint64[n[g]], host or
 *                                     device) and sums {omega, sum Y1, sum Y2, seed}
 *                                     (host uint64[4]); any may be NULL */
lap_status lap_batch_ecc(lap_batch *b, double *out, int on_device);
lap_status lap_batch_ldiag(lap_batch *b, double *out, int on_device);
lap_status lap_batch_kemeny(lap_batch *b, double *out);
lap_status lap_batch_completion(lap_batch *b, double *seconds);
/* Per graph: Tr(L^+) (the Kirchhoff index as Section 5 defines it), host double[n_graphs]. */
lap_status lap_batch_kirchhoff(lap_batch *b, double *out);
lap_status lap_batch_counts(lap_batch *b, int32_t graph, uint64_t *cnt1, uint64_t *cnt2, uint64_t *sums,
                            int on_device);

/*
 * Single-source rows of L_v^{-1} per graph (Section 4.2, "v-absorbed walk" and
 * "loop-erased walk" lemmas), as LAP_OPT_PATH_START and lap_lv_row of a
 * lap_graph handle:
 *   lap_batch_set_path_start  start = s in [0, n[g]): from the next run on, the
 *                             first absorbed walk (or loop-included path) of
 *                             every sample of graph g starts at node s; -1
 *                             (default) restores the uniform start.  Graph g's
 *                             ECC, ldiag and Kirchhoff outputs are then not
 *                             estimates; its Wilson counts and Kemeny's
 *                             constant are unchanged.  Synchronises.
 *   lap_batch_lv_row          out[u] = cnt2[u] / (omega d_u) for graph g
 *                             (double[n[g]], host or device): row s of L_v^{-1}
 *                             with a fixed start, y2(u) of Alg. 2 without.
 */
lap_status lap_batch_set_path_start(lap_batch *b, int32_t graph, int32_t start);
lap_status lap_batch_lv_row(lap_batch *b, int32_t graph, double *out, int on_device);

/* Graph g's node count, arc count, root and node offset in the result arrays. */
lap_status lap_batch_graph_info(const lap_batch *b, int32_t graph, int32_t *n, int64_t *arcs, int32_t *root,
                                int64_t *offset);

/* Reads a lap_batch_stat_id. */
lap_status lap_batch_stat(const lap_batch *b, int32_t which, int64_t *value);

/*
 * Host-only (no device use): the work-unit queue lap_batch_run builds.
 * For n_graphs graphs with node counts n[], `order` (LAP_BOPT_ORDER values),
 * `samples` per graph and `claim` samples per unit, writes the units in claim
 * order as (unit_graph[k], unit_first[k]) for k < *n_units; cap is the room
 * in both arrays (LAP_ERR_TOO_LARGE when short; *n_units still set).
 * Largest-first and smallest-first sort graphs by n (ties: lower index first).
 */
lap_status lap_batch_schedule(int32_t n_graphs, const int32_t *n, int32_t order, uint64_t samples, uint32_t claim,
                              uint32_t *unit_graph, uint32_t *unit_first, uint64_t cap, uint64_t *n_units);

/* One-line description of the last error on this handle (b = NULL: of the
 * last failed lap_batch_create or lap_batch_schedule). */
const char *lap_batch_last_error(const lap_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* LAP_BATCH_H_ */
