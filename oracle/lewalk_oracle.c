/*
 * Oracle for the loop-erased-walk (LEWalk) estimators of
 * "Scalable Algorithms for Laplacian Pseudo-inverse Computation" (arXiv 2311.10290).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded CPU
 * statement of what the GPU library computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant generator with the CUDA library: it has its
 * own Philox, its own walk loops and its own finalize.
 *
 * What it computes, per sample id i (one "sample" = one Wilson run plus the two
 * v-absorbed walks that Alg. 2 and Alg. 4 draw alongside it):
 *
 *   (1) Wilson's LE_v process (Section 3.4; Alg. 2, the loop over j):
 *       starting from each node not yet in the tree, in the caller's order,
 *       walk until the tree is hit, recording next[u] at every step; then
 *       retrace from the walk's own start along next[] and add the
 *       loop-erased path to the tree.  Every pass of a node u counts as one
 *       visit (Lemma "Loop-erased walk interpretation": the expected number of
 *       passes of u, divided by d_u, is (L_v^{-1})_uu).
 *       Y1_i = total number of random-walk steps of the run, loops included
 *       (Alg. 4: E[Y1] = Tr((I-P_v)^{-1})).
 *   (2) One v-absorbed walk from s drawn uniformly from V (Alg. 2, the second
 *       loop over i).  Each pass of u before absorption counts into cnt2[u]
 *       (Lemma "sample the paths": E[passes of u]/d_u = (1/n) e_u^T L_v^{-1} 1).
 *   (3) One v-absorbed walk from s drawn from the stationary law pi
 *       (Alg. 4).  Y2_i = its length (E[Y2] = (1/2m) d_v^T L_v^{-1} d_v).
 *
 * Randomness: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), key = (seed_lo, seed_hi), and the
 * 64-bit value R64 = out0 | out1 << 32 of the block at counter
 *     Wilson draw at node u, its k-th draw in sample i : (u, k, i, 0)
 *     uniform-start walk, sample i, step t (t=0: start): (t, 0, i, 1)
 *     pi-start walk,      sample i, step t (t=0: start): (t, 0, i, 2)
 * A uniform integer in [0, r) is the high 64 bits of R64 * r.  Keying the
 * Wilson draws by (node, draw index) makes every draw an entry of Wilson's
 * per-node stack (Section 3.4, stack representation), so the counts do not
 * depend on the order in which start nodes are taken.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- Philox */

/* Philox4x32 with 10 rounds as defined in SC'11: each round multiplies
 * words 0 and 2 by the two round multipliers, swaps the word pairs and xors
 * the high halves with the round key; the key is bumped by the two Weyl
 * constants between rounds. */
static void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Exported for the known-answer test. */
void oracle_philox_block(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    oracle_philox4x32_10(ctr, key, out);
}

static uint64_t oracle_r64(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    oracle_philox4x32_10(ctr, key, out);
    return (uint64_t)out[0] | ((uint64_t)out[1] << 32);
}

/* Uniform integer in [0, r): high word of the 128-bit product. */
static uint64_t oracle_below(uint64_t x, uint64_t r)
{
    return (uint64_t)(((unsigned __int128)x * (unsigned __int128)r) >> 64);
}

/* RandomNeighbor(u) of Alg. 2 for a given 64-bit random value. */
static int32_t oracle_neighbor(const int32_t *row_ptr, const int32_t *col, int32_t u, uint64_t x)
{
    int64_t d = (int64_t)row_ptr[u + 1] - row_ptr[u];
    return col[row_ptr[u] + (int64_t)oracle_below(x, (uint64_t)d)];
}

/* --------------------------------------------------------- one sample id */

/* Runs sample id i and adds its counts.  visits[] and next[] are caller
 * scratch of n entries; intree[] of n bytes.  order: the n-1 (or n; v is
 * skipped) start nodes in the order Alg. 2 takes them; NULL means id order.
 * Returns 0, or -1 if the step budget (max_steps, 0 = none) ran out. */
/* Control-variate sums (all optional, NULL = off): with integer potentials
 * h1[n], h2[n] and S1[u] = sum of h1 over N(u), S2 likewise,
 *   a1[u] += h1[w] for every Wilson draw at u choosing w,
 *   a2[u] += h2[w] and p2[u] += 1 for every pi-walk step at u choosing w,
 *   *m2_out = sum over the pi-walk steps of (d_u h2[w] - S2[u]) / d_u.
 * Each increment d_u h[w] - S[u] has mean zero given u, because
 * sum over w in N(u) of (d_u h[w] - S[u]) = d_u S[u] - d_u S[u] = 0. */
typedef struct {
    const int64_t *h1, *h2, *S1, *S2;
    int64_t *a1, *a2, *p2;
} oracle_cv;

/* paths = 0: the two v-absorbed walks take their own draws (stream 1 for the
 * uniform start, stream 2 for the pi start), as Alg. 2 and Alg. 4 print them.
 * paths = 1: they are the loop-included paths of the sample's own stacks
 * (Section 4.2, "loop-erased walk" interpretation and "Sample from the
 * paths"; Section 5.2): same start draws, and the j-th departure of a path
 * from u takes stack entry j of u, i.e. draw (u, j, i, 0) of the Wilson run.
 * path_start >= 0: the first absorbed walk (or path) starts at that node
 * instead of a uniform draw; its passes then estimate row path_start of
 * L_v^{-1} (Section 4.2, "v-absorbed walk" and "loop-erased walk" lemmas:
 * (L_v^{-1})_{su} = E[passes of u on a walk from s] / d_u). */
static int oracle_one_sample(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t v,
                             uint64_t seed, uint32_t i, const int32_t *order, int32_t n_order,
                             uint32_t *draws, int32_t *next, uint8_t *intree,
                             uint64_t *cnt1, uint64_t *cnt2,
                             uint64_t *y1_out, uint64_t *y2_out, int32_t *tree_out,
                             uint64_t max_steps, const oracle_cv *cv, double *m2_out, int paths,
                             int32_t path_start)
{
    /* Alg. 2: InTree[u] = false, Next[u] = -1 for all u; InTree[v] = true. */
    for (int32_t u = 0; u < n; ++u) { intree[u] = 0; next[u] = -1; draws[u] = 0; }
    intree[v] = 1;

    uint64_t y1 = 0;
    int32_t count = order ? n_order : n;
    for (int32_t j = 0; j < count; ++j) {
        int32_t s = order ? order[j] : j;
        if (s == v) continue;
        /* Walk from s until the tree is hit; every pass is a visit. */
        int32_t u = s;
        while (!intree[u]) {
            cnt1[u] += 1;
            y1 += 1;
            if (max_steps && y1 > max_steps) return -1;
            uint64_t x = oracle_r64(seed, (uint32_t)u, draws[u], i, 0u);
            draws[u] += 1;
            next[u] = oracle_neighbor(row_ptr, col, u, x);
            if (cv && cv->h1) cv->a1[u] += cv->h1[next[u]];
            u = next[u];
        }
        /* Retrace from the walk's own start: the loop-erased path joins the tree. */
        u = s;
        while (!intree[u]) {
            intree[u] = 1;
            u = next[u];
        }
    }
    if (tree_out)
        for (int32_t u = 0; u < n; ++u) tree_out[u] = (u == v) ? -1 : next[u];

    /* v-absorbed walk from a uniformly drawn s (Alg. 2), or the sample's
     * loop-included path from s.  draws[] now counts a path's departures. */
    {
        uint64_t t = 0;
        int32_t u = path_start >= 0 ? path_start
                                    : (int32_t)oracle_below(oracle_r64(seed, 0u, 0u, i, 1u), (uint64_t)n);
        if (paths)
            for (int32_t w = 0; w < n; ++w) draws[w] = 0;
        while (u != v) {
            cnt2[u] += 1;
            t += 1;
            if (max_steps && t > max_steps) return -1;
            if (paths) {
                uint64_t x = oracle_r64(seed, (uint32_t)u, draws[u], i, 0u);
                draws[u] += 1;
                u = oracle_neighbor(row_ptr, col, u, x);
            } else {
                u = oracle_neighbor(row_ptr, col, u, oracle_r64(seed, (uint32_t)t, 0u, i, 1u));
            }
        }
    }
    /* v-absorbed walk from s ~ pi (Alg. 4): the head of a uniformly drawn arc
     * is distributed as pi(w) = d_w / 2m. */
    uint64_t y2 = 0;
    double m2 = 0.0;
    {
        int64_t arcs = row_ptr[n];
        int32_t u = col[oracle_below(oracle_r64(seed, 0u, 0u, i, 2u), (uint64_t)arcs)];
        if (paths)
            for (int32_t w = 0; w < n; ++w) draws[w] = 0;
        while (u != v) {
            y2 += 1;
            if (max_steps && y2 > max_steps) return -1;
            int32_t w;
            if (paths) {
                uint64_t x = oracle_r64(seed, (uint32_t)u, draws[u], i, 0u);
                draws[u] += 1;
                w = oracle_neighbor(row_ptr, col, u, x);
            } else {
                w = oracle_neighbor(row_ptr, col, u, oracle_r64(seed, (uint32_t)y2, 0u, i, 2u));
            }
            if (cv && cv->h2) {
                int64_t d = (int64_t)row_ptr[u + 1] - row_ptr[u];
                cv->a2[u] += cv->h2[w];
                cv->p2[u] += 1;
                m2 += (double)(d * cv->h2[w] - cv->S2[u]) / (double)d;
            }
            u = w;
        }
    }
    if (m2_out) *m2_out = m2;
    *y1_out = y1;
    *y2_out = y2;
    return 0;
}

/*
 * Samples ids first .. first+count-1 and ADDS to cnt1[n], cnt2[n].
 * y1[count], y2[count] (optional) receive the per-sample Y1, Y2;
 * tree[count*n] (optional) receives each sample's parent array (-1 at v).
 * Returns 0 on success, -1 on a step-budget overrun, -2 on bad arguments.
 */
int oracle_sample(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t v,
                  uint64_t seed, uint64_t first, uint64_t count,
                  const int32_t *order, int32_t n_order,
                  uint64_t *cnt1, uint64_t *cnt2,
                  uint64_t *y1, uint64_t *y2, int32_t *tree, uint64_t max_steps, int paths,
                  int32_t path_start)
{
    if (n <= 0 || v < 0 || v >= n || first + count > 0x100000000ull || path_start >= n) return -2;
    uint32_t *draws = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    int32_t *next = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint8_t *intree = (uint8_t *)malloc((size_t)n);
    if (!draws || !next || !intree) { free(draws); free(next); free(intree); return -2; }
    int rc = 0;
    for (uint64_t q = 0; q < count; ++q) {
        uint64_t a = 0, b = 0;
        rc = oracle_one_sample(n, row_ptr, col, v, seed, (uint32_t)(first + q), order, n_order,
                               draws, next, intree, cnt1, cnt2, &a, &b,
                               tree ? tree + (size_t)q * (size_t)n : NULL, max_steps, NULL, NULL, paths,
                               path_start);
        if (rc) break;
        if (y1) y1[q] = a;
        if (y2) y2[q] = b;
    }
    free(draws); free(next); free(intree);
    return rc;
}

/*
 * oracle_sample with the control-variate sums (see oracle_cv): potentials
 * h1 (Wilson draws) and h2 (pi walk), either may be NULL.  a1, a2, p2 are
 * ADDED to; m2[count] (optional) receives the per-sample pi-walk martingale.
 */
int oracle_sample_cv(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t v,
                     uint64_t seed, uint64_t first, uint64_t count,
                     uint64_t *cnt1, uint64_t *cnt2, uint64_t *y1, uint64_t *y2,
                     const int64_t *h1, const int64_t *h2, int64_t *a1, int64_t *a2, int64_t *p2, double *m2,
                     int paths)
{
    if (n <= 0 || v < 0 || v >= n || first + count > 0x100000000ull) return -2;
    int64_t *S1 = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *S2 = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    uint32_t *draws = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    int32_t *next = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint8_t *intree = (uint8_t *)malloc((size_t)n);
    for (int32_t u = 0; u < n; ++u)
        for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            if (h1) S1[u] += h1[col[e]];
            if (h2) S2[u] += h2[col[e]];
        }
    oracle_cv cv = {h1, h2, S1, S2, a1, a2, p2};
    int rc = 0;
    for (uint64_t q = 0; q < count; ++q) {
        uint64_t a = 0, b = 0;
        double mm = 0.0;
        rc = oracle_one_sample(n, row_ptr, col, v, seed, (uint32_t)(first + q), NULL, 0,
                               draws, next, intree, cnt1, cnt2, &a, &b, NULL, 0, &cv, &mm, paths, -1);
        if (rc) break;
        if (y1) y1[q] = a;
        if (y2) y2[q] = b;
        if (m2) m2[q] = mm;
    }
    free(S1); free(S2); free(draws); free(next); free(intree);
    return rc;
}

/*
 * Hitting-time targets (Section 3.2, v-absorbed walk lemma: the expected
 * length of a walk from u absorbed at v is h(u, v) = (L_v^{-1} d)_u).  For
 * every node u and repetition r in [0, reps), one walk from u until v; step t
 * (t = 1, 2, ...) uses Philox counter (t, u, r, 3).  sums[u] += total length.
 */
int oracle_hitting_walks(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t v,
                         uint64_t seed, uint32_t reps, uint64_t *sums, uint64_t max_steps)
{
    if (n <= 0 || v < 0 || v >= n) return -2;
    for (int32_t u = 0; u < n; ++u) {
        for (uint32_t r = 0; r < reps; ++r) {
            uint64_t t = 0;
            int32_t x = u;
            while (x != v) {
                t += 1;
                if (max_steps && t > max_steps) return -1;
                x = oracle_neighbor(row_ptr, col, x, oracle_r64(seed, (uint32_t)t, (uint32_t)u, r, 3u));
            }
            sums[u] += t;
        }
    }
    return 0;
}

/*
 * Cycle popping on Wilson's stacks (Section 3.4, stack representation): the
 * top of S[u] is the draw (u, pops[u], i, 0).  While the top-pointer graph on
 * the non-tree nodes has nodes whose top path reaches the tree, those paths
 * join the tree; the rest of that graph is made of cycles with paths feeding
 * them, and every cycle is popped (each of its nodes moves to its next stack
 * entry).  Wilson's theorem says the popped cycles, and so pops[u], do not
 * depend on the order of popping; the number of visits of u in the sequential
 * run equals pops[u] + 1.  Only cnt1, Y1 and the tree are produced here (the
 * absorbed walks are unchanged), so tests can compare them with
 * oracle_sample.
 */
int oracle_cyclepop(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t v,
                    uint64_t seed, uint64_t first, uint64_t count,
                    uint64_t *cnt1, uint64_t *y1, int32_t *tree)
{
    if (n <= 0 || v < 0 || v >= n) return -2;
    uint32_t *pops = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    int32_t *top = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint8_t *state = (uint8_t *)malloc((size_t)n);   /* 0 undecided, 1 tree */
    int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!pops || !top || !state || !mark) { free(pops); free(top); free(state); free(mark); return -2; }
    for (uint64_t q = 0; q < count; ++q) {
        uint32_t i = (uint32_t)(first + q);
        for (int32_t u = 0; u < n; ++u) {
            pops[u] = 0; state[u] = 0;
            if (u != v) top[u] = oracle_neighbor(row_ptr, col, u, oracle_r64(seed, (uint32_t)u, 0u, i, 0u));
        }
        state[v] = 1; top[v] = -1;
        int32_t remaining = n - 1;
        while (remaining > 0) {
            /* Nodes whose top path reaches the tree join it. */
            int changed = 1;
            while (changed) {
                changed = 0;
                for (int32_t u = 0; u < n; ++u)
                    if (!state[u] && state[top[u]]) { state[u] = 1; --remaining; changed = 1; }
            }
            if (remaining == 0) break;
            /* Every remaining node leads into a cycle: find each cycle by
             * following tops with a per-start stamp, then pop it. */
            for (int32_t u = 0; u < n; ++u) mark[u] = -1;
            int32_t *cyc = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
            int32_t ncyc = 0;
            for (int32_t s = 0; s < n; ++s) {
                if (state[s] || mark[s] != -1) continue;
                int32_t u = s;
                while (!state[u] && mark[u] == -1) { mark[u] = s; u = top[u]; }
                if (!state[u] && mark[u] == s) {
                    /* u is on a cycle first met from s. */
                    int32_t w = u;
                    do { cyc[ncyc++] = w; w = top[w]; } while (w != u);
                }
            }
            for (int32_t c = 0; c < ncyc; ++c) {
                int32_t u = cyc[c];
                pops[u] += 1;
                top[u] = oracle_neighbor(row_ptr, col, u, oracle_r64(seed, (uint32_t)u, pops[u], i, 0u));
            }
            free(cyc);
        }
        uint64_t total = 0;
        for (int32_t u = 0; u < n; ++u) {
            if (u == v) continue;
            cnt1[u] += (uint64_t)pops[u] + 1u;
            total += (uint64_t)pops[u] + 1u;
        }
        if (y1) y1[q] = total;
        if (tree)
            for (int32_t u = 0; u < n; ++u) tree[(size_t)q * (size_t)n + (size_t)u] = (u == v) ? -1 : top[u];
    }
    free(pops); free(top); free(state); free(mark);
    return 0;
}

/* ------------------------------------------------------------- finalize */

/* Neumaier-compensated sum, so the oracle's totals are accurate to about one
 * rounding whatever n is. */
static double oracle_sum(const double *x, int32_t n)
{
    double s = 0.0, c = 0.0;
    for (int32_t k = 0; k < n; ++k) {
        double t = s + x[k];
        if ((s >= 0 ? s : -s) >= (x[k] >= 0 ? x[k] : -x[k])) c += (s - t) + x[k];
        else c += (x[k] - t) + s;
        s = t;
    }
    return s + c;
}

/*
 * Maps counts to the outputs.
 *   y1(u) = cnt1[u] / (omega d_u)           estimates (L_v^{-1})_uu      (Alg. 2)
 *   y2(u) = cnt2[u] / (omega d_u)           estimates (1/n) e_u^T L_v^{-1} 1
 *   Ldag_uu = y1(u) - 2 y2(u) + (1/n) sum_w y2(w)   for u != v   (Eq. for (L^+)_ss, Alg. 2)
 *   Ldag_vv = (1/n) sum_w y2(w)                                   (Eq. for (L^+)_vv)
 *   ecc(u)  = (n-1) / (n Ldag_uu + sum_w Ldag_ww)                 (Section 2, ECC)
 *   kemeny  = (sum Y1 - sum Y2) / omega                           (Alg. 4)
 * Any output pointer may be NULL.
 */
void oracle_finalize(int32_t n, const int32_t *row_ptr, int32_t v, uint64_t omega,
                     const uint64_t *cnt1, const uint64_t *cnt2, uint64_t sum_y1, uint64_t sum_y2,
                     double *ldiag, double *ecc, double *kemeny)
{
    double *y1 = (double *)malloc(sizeof(double) * (size_t)n);
    double *y2 = (double *)malloc(sizeof(double) * (size_t)n);
    double *ld = (double *)malloc(sizeof(double) * (size_t)n);
    double w = (double)omega;
    for (int32_t u = 0; u < n; ++u) {
        double d = (double)(row_ptr[u + 1] - row_ptr[u]);
        y1[u] = (double)cnt1[u] / (w * d);
        y2[u] = (double)cnt2[u] / (w * d);
    }
    double s2 = oracle_sum(y2, n);
    double lvv = s2 / (double)n;
    for (int32_t u = 0; u < n; ++u)
        ld[u] = (u == v) ? lvv : (y1[u] - 2.0 * y2[u]) + lvv;
    double tr = oracle_sum(ld, n);
    for (int32_t u = 0; u < n; ++u) {
        if (ldiag) ldiag[u] = ld[u];
        if (ecc) ecc[u] = (double)(n - 1) / ((double)n * ld[u] + tr);
    }
    if (kemeny) *kemeny = ((double)sum_y1 - (double)sum_y2) / w;
    free(y1); free(y2); free(ld);
}
