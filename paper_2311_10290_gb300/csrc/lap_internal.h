// Internal declarations of the GB300 library behind include/lap.h.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "lap.h"

// Device-side view of a graph: per-node row records {offset, degree} (one
// aligned 8-byte load per visit) and the column array.
struct LapDevGraph {
    const int2 *rowinfo;   // [n] {row_ptr[u], d_u}
    const int32_t *col;    // [arcs]
    int32_t n;
    int64_t arcs;
};

// Status bits written by kernels into the handle's status word.
enum : unsigned int {
    LAP_DEV_BAD_CSR = 1u,
    LAP_DEV_SELF_LOOP = 2u,
    LAP_DEV_NOT_SYMMETRIC = 4u,
    LAP_DEV_STEP_LIMIT = 8u,
    LAP_DEV_K_OVERFLOW = 16u,
    LAP_DEV_BAD_INDEX = 64u,       // a node index out of range was caught (write skipped)
};

// Accumulators of a handle on the device (one cache line).
struct LapDevAcc {
    unsigned long long sum_y1;     // sum over samples of Y1 (Wilson steps incl. loops)
    unsigned long long sum_y2;     // sum over samples of Y2 (pi-start walk length)
    unsigned int status;           // LAP_DEV_* bits
    unsigned int claim;            // next sample offset to claim inside a launch
    unsigned int ovf_count;        // compact kernel: samples withdrawn in this launch
    unsigned int pad0;
    unsigned long long pad[4];
};

// ---------------------------------------------------------------- kernels
// ingest.cu
cudaError_t lap_launch_validate(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t arcs,
                                unsigned int *status, cudaStream_t st);
cudaError_t lap_launch_rowinfo(const int32_t *row_ptr, int32_t n, int2 *rowinfo, cudaStream_t st);
cudaError_t lap_launch_argmax_degree(const int2 *rowinfo, int32_t n, unsigned long long *best, cudaStream_t st);
cudaError_t lap_launch_bfs_init(int32_t *hops, int32_t n, int32_t root, cudaStream_t st);
cudaError_t lap_launch_bfs_level(const int2 *rowinfo, const int32_t *col, int32_t *hops, int32_t n,
                                 int32_t level, unsigned int *found, cudaStream_t st);

// sampler.cu
struct LapSampleLaunch {
    LapDevGraph g;
    int32_t root;
    uint64_t seed;
    uint32_t first;          // first sample id of this launch
    uint32_t count;          // samples in this launch
    uint64_t slots;          // lanes with their own Wilson state
    void *ws;                // slots * n * 8 bytes
    unsigned int *slot_epoch;
    unsigned long long *rep1;
    unsigned long long *cnt2;
    LapDevAcc *acc;
    uint64_t step_limit;
    int block;                   // threads per block; 0 = pick_block()
    int num_sms;
    unsigned long long *y1_out;  // optional [count]: Y1 of sample first+q at q
    unsigned long long *y2_out;  // optional [count]: Y2 of sample first+q at q
    uint64_t slot_bytes;         // compact kernel: bytes of one slot (state + stack)
    uint64_t n_pad;              // compact kernel: state bytes of one slot (n rounded up to 256)
    uint32_t stack_cap;          // compact kernel: stack entries of one slot
    uint32_t tbl_log2;           // compact kernel: log2 of the count-table entries
    uint32_t paths;              // 1: the absorbed walks are the loop-included paths of the sample's
                                 // own stacks (departure j from u takes draw (u, j, i, 0)); 0: own draws
    unsigned int *ovf_ids;       // compact kernel: withdrawn sample ids [count]
    const unsigned int *ids;     // wide kernel: explicit sample ids [count] (NULL: first + q)
    uint32_t trace_base;         // wide kernel with ids: y1_out/y2_out index = id - trace_base
    // Control variate (NULL pointers: off).  Wilson draws at u choosing w add
    // h1[w] to a1[u]; pi-walk steps at u choosing w add h2[w] to a2[u] and 1
    // to p2[u], and (d_u h2[w] - S2[u]) / d_u to the sample's M2.
    const long long *cv_h1;
    unsigned long long *cv_a1;
    const long long *cv_h2;
    const long long *cv_S2;
    unsigned long long *cv_a2;
    unsigned long long *cv_p2;
    double *m2_out;              // optional [count]: per-sample M2 (with y1_out)
    uint32_t flags;              // wide kernel: LAP_SAMPLE_* below
    uint32_t ustart;             // 0: the first absorbed walk (or path) starts at a uniform draw
                                 // (Alg. 2); s + 1: it starts at node s (single-source rows of L_v^{-1})
};
enum : uint32_t {
    LAP_SAMPLE_ONE_PER_LANE = 1u,   // lane j runs exactly sample first + j (j < count), so its
                                    // slot ends holding that sample's tree (Next of every node)
    LAP_SAMPLE_WILSON_ONLY = 2u,    // skip the two absorbed walks (Y2 = 0, no cnt2 passes)
};
cudaError_t lap_launch_sample(const LapSampleLaunch &p, cudaStream_t st);
// sampler_compact.cu
cudaError_t lap_launch_sample_compact(const LapSampleLaunch &p, cudaStream_t st);
// sampler_group.cu: `walkers` lanes per sample (2, 4, 8 or 16); p.slots counts groups;
// p.stack_cap is the stack capacity of each walker
cudaError_t lap_launch_sample_group(const LapSampleLaunch &p, int walkers, cudaStream_t st);

// ------------------------------------------------------------ batches
// One graph of a batch (device descriptor).  Pointers index the batch's
// packed arenas; row records hold offsets local to the graph's columns.
struct LapBatchGraph {
    const int2 *rowinfo;          // [n]
    const int32_t *col;           // [arcs]
    unsigned long long *rep1;     // [n] repeat Wilson visits
    unsigned long long *cnt2;     // [n] uniform-start walk passes
    double *ldiag;                // [n] finalize output
    double *ecc;                  // [n] finalize output
    int64_t arcs;
    uint64_t step_limit;
    int32_t n;
    int32_t root;
    uint32_t count;               // samples of the graph in the current run
    uint32_t ustart;              // as LapSampleLaunch::ustart, for this graph
};

// Control block of a batch launch (one cache line).
struct LapBatchCtl {
    unsigned long long t0;        // globaltimer at kernel start (minimum over blocks)
    unsigned long long steps;     // probe launches: walk steps taken before the deadline
    unsigned int claim;           // next work unit
    unsigned int status;          // LAP_DEV_* bits
    unsigned int ovf_count;       // samples withdrawn (re-run with the 8-byte kernel)
    unsigned int pad[9];
};

struct LapBatchLaunch {
    const LapBatchGraph *graphs;
    const uint2 *units;           // work units {graph, first sample}, in claim order
    uint32_t n_units;
    uint32_t claim;               // samples per unit (the last unit of a graph may hold fewer)
    uint64_t seed;
    uint64_t lanes;
    void *ws;                     // lanes * slot_bytes
    uint64_t slot_bytes;
    uint64_t n_pad;               // state bytes of a slot (largest n rounded up to 256)
    uint32_t stack_cap;
    uint32_t tbl_log2;            // log2 of the count-table entries of a slot
    uint32_t paths;               // as LapSampleLaunch::paths
    unsigned int *slot_meta;      // per lane: bit 31 epoch, bits 0..30 extent of bytes carrying it
    LapDevAcc *acc;               // [graphs] sum Y1, sum Y2
    unsigned int *done;           // [graphs] samples finished
    unsigned long long *t_done;   // [graphs] globaltimer when the graph's last sample finished
    LapBatchCtl *ctl;
    uint2 *ovf;                   // [ovf_cap] withdrawn samples {graph, sample id}
    uint32_t ovf_cap;
    unsigned long long window_ns; // probe launches: each lane stops after this long
    int block;
    int num_sms;
};
// sampler_batch.cu
cudaError_t lap_launch_batch(const LapBatchLaunch &p, bool probe, cudaStream_t st);
int lap_batch_block(const LapBatchLaunch &p);
uint64_t lap_batch_resident_lanes(int block, int num_sms);
// solve.cu: conjugate gradients for L_v x = b; scratch: 4 n + 2 * 1024 + 8 doubles
cudaError_t lap_run_lv_solve(const int2 *rowinfo, const int32_t *col, int32_t n, int32_t v, const double *b, double *x,
                             double *scratch, double rtol, int32_t maxiter, int32_t *iterations, double *residual,
                             cudaStream_t st);

// finalize.cu: finalize of every graph of a batch, bit-identical per graph to
// lap_launch_finalize; red holds graphs * (1024 + 2) doubles.
cudaError_t lap_launch_finalize_batch(const LapBatchGraph *graphs, int32_t n_graphs, int32_t max_n, uint64_t omega,
                                      double *red, cudaStream_t st);

// ------------------------------------------------------------ SpanTree (Alg. 1, Alg. 3)
struct LapSpanTreeLaunch {
    const int2 *rowinfo;
    const int32_t *bpar;                 // [n] BFS parent (-1 at the root)
    const unsigned long long *trees;     // count slots of n 8-byte Wilson states (low 32 bits: Next)
    int32_t n;
    int32_t root;
    uint32_t count;                      // trees in this launch
    int32_t *scratch;                    // blocks * scratch_ints
    uint64_t scratch_ints;
    unsigned long long *x1, *x2, *x2d;   // [n] integer sums over trees
    unsigned int *status;
};
// spantree.cu
cudaError_t lap_launch_bfs_parent(const int2 *rowinfo, const int32_t *col, const int32_t *hops, int32_t n, int32_t root,
                                  int32_t *bpar, unsigned int *status, cudaStream_t st);
uint64_t lap_spantree_scratch_ints(int32_t n);
cudaError_t lap_launch_spantree(const LapSpanTreeLaunch &p, int blocks, cudaStream_t st);
cudaError_t lap_launch_spantree_finalize(const int2 *rowinfo, int32_t n, int32_t root, uint64_t omega,
                                         const long long *X1, const long long *X2, const long long *X2d,
                                         double *ldiag, double *ecc, double *red, cudaStream_t st);

// Threads per block for `lanes` persistent lanes: the smallest warp multiple
// (up to 256) that keeps at most 16 blocks per SM, so that the blocks, and
// the lanes with them, spread evenly over all SMs.
inline int lap_pick_block(uint64_t lanes, int num_sms)
{
    int block = 32;
    const uint64_t sms = num_sms > 0 ? (uint64_t)num_sms : 1ull;
    while (block < 256 && lanes > 16ull * sms * (uint64_t)block) block *= 2;
    return block;
}

enum LapKernel : int { LAP_KERNEL_WIDE = 1, LAP_KERNEL_COMPACT = 2, LAP_KERNEL_GROUP = 3 };

// Compact kernels: log2 of the entries of the per-lane table of draw counts
// above 30 (after the path stack; see compact_state.cuh): the next power of
// two >= n, from 2^8 to 2^13 entries (8 bytes each).
inline uint32_t lap_table_log2(int64_t n)
{
    uint32_t l = 8;
    while (l < 13 && (1ll << l) < n) ++l;
    return l;
}

// Control variate (cv.cu, mlp.cu).
constexpr int LAP_CV_FIXED_POINT_BITS = 16;   // h = round(2^16 phi)
constexpr int LAP_CV_ABSORB_ITERS = 8;        // feature f7: P(hit v within 8 steps)
cudaError_t lap_launch_features(const int2 *rowinfo, const int32_t *col, const int32_t *hops, int32_t n, int32_t root,
                                double *scratch, float *feat, cudaStream_t st);
cudaError_t lap_launch_potential(const int2 *rowinfo, const int32_t *col, int32_t n, const double *phi, long long *h,
                                 long long *S, cudaStream_t st);
cudaError_t lap_launch_hitting_walks(const LapDevGraph &g, int32_t root, uint64_t seed, uint32_t reps, uint64_t limit,
                                     unsigned long long *sums, unsigned int *status, int num_sms, cudaStream_t st);
cudaError_t lap_launch_cv_finalize(const int2 *rowinfo, int32_t n, int32_t root, uint64_t omega,
                                   const unsigned long long *rep1, const unsigned long long *cnt2,
                                   const long long *a1, const long long *S1, double beta1,
                                   const long long *a2, const long long *p2, const long long *S2,
                                   double *ldiag, double *ecc, double *red, double *m2_out, cudaStream_t st);
cudaError_t lap_launch_cv_targets(int32_t n, int32_t root, uint64_t omega, const unsigned long long *rep1,
                                  const unsigned long long *hit, uint32_t reps, double mean_y2, float *targets,
                                  cudaStream_t st);
cudaError_t lap_launch_cv_potentials(const int2 *rowinfo, int32_t n, int32_t root, const float *y, double scale2,
                                     double *phi1, double *phi2, cudaStream_t st);
cudaError_t lap_launch_beta1_batch(const int2 *rowinfo, int32_t n, int32_t root, uint64_t omega,
                                   const unsigned long long *rep1, const long long *a1, const long long *S1,
                                   long long *prev_c1, long long *prev_a1, double *vb, double *zb, cudaStream_t st);
cudaError_t lap_launch_beta1_reduce(int32_t n, int32_t batches, const double *vb, const double *zb, double *red,
                                    double *out, cudaStream_t st);
cudaError_t lap_launch_beta2_reduce(const unsigned long long *y1, const unsigned long long *y2, const double *m2,
                                    int64_t count, double *red, double *out, cudaStream_t st);
// MLP forward (T = nullptr) or loss and gradient: mlp_tc.cu (tcgen05, TMEM
// accumulators) or mlp.cu (mma.sync), per lap_mlp_select.
cudaError_t lap_launch_mlp_tc(const float *P, const float *X, const float *T, int64_t n, float wk0, float wk1,
                              float *Y, float *G, float *loss, cudaStream_t st);
cudaError_t lap_launch_mlp_mma_sync(const float *P, const float *X, const float *T, int64_t n, float wk0,
                                    float wk1, float *Y, float *G, float *loss, cudaStream_t st);
cudaError_t lap_launch_adamw(float *w, float *m, float *v, const float *g, int64_t count, int32_t step, float lr,
                             float b1, float b2, float eps, float wd, cudaStream_t st);

// finalize.cu
cudaError_t lap_launch_finalize(const int2 *rowinfo, int32_t n, int32_t root, uint64_t omega,
                                const unsigned long long *rep1, const unsigned long long *cnt2,
                                double *ldiag, double *ecc, double *red, cudaStream_t st);
cudaError_t lap_launch_rw_betweenness(int32_t n, const double *ldiag, const double *red, double *out, cudaStream_t st);
cudaError_t lap_launch_lv_row(const int2 *rowinfo, int32_t n, uint64_t omega, const unsigned long long *cnt2,
                              double *out, cudaStream_t st);
cudaError_t lap_launch_counts(int32_t n, int32_t root, uint64_t omega, const unsigned long long *rep1,
                              unsigned long long *cnt1, cudaStream_t st);
cudaError_t lap_launch_rep_from_counts(int32_t n, int32_t root, uint64_t omega, const unsigned long long *cnt1,
                                       unsigned long long *rep1, unsigned int *bad, cudaStream_t st);

struct lap_graph {
    int device = 0;
    int num_sms = 0;
    int32_t n = 0;
    int64_t arcs = 0;

    int32_t *d_row_ptr = nullptr;
    int32_t *d_col = nullptr;
    int2 *d_rowinfo = nullptr;
    int32_t *d_hops = nullptr;
    unsigned long long *d_rep1 = nullptr;   // repeat visits per node (visits - 1, summed)
    unsigned long long *d_cnt2 = nullptr;   // uniform-start walk passes per node
    LapDevAcc *d_acc = nullptr;
    double *d_ldiag = nullptr;
    double *d_ecc = nullptr;
    double *d_red = nullptr;                // reduction scratch
    double *d_aux = nullptr;                // [n] random-walk betweenness, lap_lv_row (allocated on first use)
    unsigned int *d_slot_epoch = nullptr;   // per-slot epoch parity of the Wilson state
    uint64_t slot_epoch_cap = 0;

    cudaStream_t stream = nullptr;
    int32_t root = -1;
    uint64_t seed = 0;
    bool seed_set = false;
    uint64_t omega = 0;                     // samples drawn since lap_set_root
    uint64_t cursor = 0;                    // next sample id
    bool results_valid = false;

    void *ws = nullptr;                     // Wilson state workspace
    uint64_t ws_bytes = 0;
    bool ws_owned = false;
    bool ws_zeroed = false;

    uint64_t step_limit = 0;                // 0: default
    uint64_t slots_opt = 0;
    int block_opt = 0;
    int kernel_opt = 0;                     // 0 auto, LAP_KERNEL_WIDE, LAP_KERNEL_COMPACT, LAP_KERNEL_GROUP
    int walkers = 0;                        // LAP_OPT_WALKERS (kernel 3; 0 = automatic)
    uint32_t paths_opt = 0;                 // LAP_OPT_PATHS
    int32_t path_start = -1;                // LAP_OPT_PATH_START (-1: uniform start)
    uint32_t stack_cap = 0;                 // 0: default, about 16 sqrt(n)
    int last_kernel = 0;                    // layout the workspace currently holds
    int used_kernel = 0;                    // kernel of the last lap_sample call (LAP_STAT_LAST_KERNEL)
    bool compact_disabled = false;          // set after a compact launch overflowed
    int64_t fallbacks = 0;

    // Control variate.
    long long *d_cv_h1 = nullptr, *d_cv_S1 = nullptr, *d_cv_h2 = nullptr, *d_cv_S2 = nullptr;
    unsigned long long *d_cv_a1 = nullptr, *d_cv_a2 = nullptr, *d_cv_p2 = nullptr;
    double *d_feat_scratch = nullptr;
    bool cv1 = false, cv2 = false;

    // SpanTree estimators (allocated on first use).
    int32_t *d_bpar = nullptr;
    bool bpar_valid = false;
    unsigned long long *d_st_x1 = nullptr, *d_st_x2 = nullptr, *d_st_x2d = nullptr, *d_st_rep1 = nullptr;
    double *d_st_ldiag = nullptr, *d_st_ecc = nullptr, *d_st_red = nullptr;
    LapDevAcc *d_st_acc = nullptr;
    int32_t *d_st_scratch = nullptr;
    int st_blocks = 0;
    uint64_t st_omega = 0, st_cursor = 0, st_seed = 0;
    bool st_seed_set = false;

    // Samples a compact launch withdrew; re-run with the wide kernel.
    unsigned int *d_ovf_ids = nullptr;
    uint64_t ovf_cap = 0;
    bool pending = false;
    LapSampleLaunch pending_launch;

    lap_status sticky = LAP_OK;
    std::string err;
};
