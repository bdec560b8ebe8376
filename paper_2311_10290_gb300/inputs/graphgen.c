/*
 * Seeded synthetic graph generators: the inputs shared by the GPU library's
 * tests/benchmarks and by the CPU oracle.  Nothing here computes any part of
 * the sampling method; it only produces undirected, unweighted CSR graphs.
 *
 * Output format (what the method assumes, Section 2 of the paper): CSR with
 * int32 row_ptr[n+1] and col[2m], every edge stored in both directions, rows
 * sorted ascending, no self-loops, no duplicate edges.  When `lcc` is set the
 * graph is reduced to its largest connected component, with the kept nodes
 * relabelled 0..n'-1 in increasing original id.
 *
 * Randomness is SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014); it is unrelated to the
 * Philox streams the samplers use.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t n;          /* nodes after cleaning */
    int64_t arcs;       /* = 2m */
    int32_t *row_ptr;   /* n + 1 */
    int32_t *col;       /* arcs */
    int32_t *orig_id;   /* n: id of each node before the LCC relabel */
} gg_graph;

typedef struct { uint64_t s; } gg_rng;

static uint64_t gg_next(gg_rng *r)
{
    uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static double gg_unif(gg_rng *r) { return (double)(gg_next(r) >> 11) * (1.0 / 9007199254740992.0); }
static uint64_t gg_below(gg_rng *r, uint64_t k) { return (uint64_t)(((unsigned __int128)gg_next(r) * k) >> 64); }

static int gg_bits(int64_t n)
{
    int b = 1;
    while (((int64_t)1 << b) < n) ++b;
    return b;
}

/* LSD radix sort of 64-bit keys that use the low `bits` bits. */
static int gg_radix(uint64_t *a, int64_t len, int bits)
{
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(len > 0 ? len : 1));
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * 65536);
    if (!tmp || !cnt) { free(tmp); free(cnt); return -1; }
    uint64_t *src = a, *dst = tmp;
    for (int shift = 0; shift < bits; shift += 16) {
        memset(cnt, 0, sizeof(int64_t) * 65536);
        for (int64_t k = 0; k < len; ++k) cnt[(src[k] >> shift) & 0xFFFF]++;
        int64_t acc = 0;
        for (int b = 0; b < 65536; ++b) { int64_t c = cnt[b]; cnt[b] = acc; acc += c; }
        for (int64_t k = 0; k < len; ++k) dst[cnt[(src[k] >> shift) & 0xFFFF]++] = src[k];
        uint64_t *t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, sizeof(uint64_t) * (size_t)len);
    free(tmp); free(cnt);
    return 0;
}

static int32_t gg_find(int32_t *par, int32_t x)
{
    while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; }
    return x;
}

/* Sorted, de-duplicated arc keys (u << sh | w) -> CSR graph (optionally LCC). */
static gg_graph *gg_keys_to_graph(int32_t n, uint64_t *keys, int64_t len, int sh, int lcc)
{
    uint64_t mask = ((uint64_t)1 << sh) - 1;
    int32_t *keepmap = NULL;
    int32_t n2 = n;
    int32_t *orig = NULL;
    if (lcc) {
        int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        for (int32_t u = 0; u < n; ++u) par[u] = u;
        for (int64_t k = 0; k < len; ++k) {
            int32_t a = gg_find(par, (int32_t)(keys[k] >> sh)), b = gg_find(par, (int32_t)(keys[k] & mask));
            if (a != b) { if (a < b) par[b] = a; else par[a] = b; }
        }
        int32_t *size = (int32_t *)calloc((size_t)n, sizeof(int32_t));
        for (int32_t u = 0; u < n; ++u) size[gg_find(par, u)]++;
        int32_t best = 0;
        for (int32_t u = 0; u < n; ++u) if (size[u] > size[best]) best = u;   /* ties: smallest root id */
        keepmap = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        n2 = 0;
        for (int32_t u = 0; u < n; ++u) keepmap[u] = (gg_find(par, u) == best) ? n2++ : -1;
        orig = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n2 > 0 ? n2 : 1));
        for (int32_t u = 0; u < n; ++u) if (keepmap[u] >= 0) orig[keepmap[u]] = u;
        free(par); free(size);
    } else {
        orig = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        for (int32_t u = 0; u < n; ++u) orig[u] = u;
    }
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    g->n = n2;
    g->orig_id = orig;
    g->row_ptr = (int32_t *)calloc((size_t)n2 + 1, sizeof(int32_t));
    int64_t arcs = 0;
    for (int64_t k = 0; k < len; ++k) {
        int32_t u = (int32_t)(keys[k] >> sh);
        if (!keepmap || keepmap[u] >= 0) arcs++;
    }
    g->arcs = arcs;
    g->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(arcs > 0 ? arcs : 1));
    int64_t e = 0;
    for (int64_t k = 0; k < len; ++k) {
        int32_t u = (int32_t)(keys[k] >> sh), w = (int32_t)(keys[k] & mask);
        if (keepmap) { if (keepmap[u] < 0) continue; u = keepmap[u]; w = keepmap[w]; }
        g->row_ptr[u + 1]++;
        g->col[e++] = w;           /* relabelling is monotone: rows stay sorted */
    }
    for (int32_t u = 0; u < n2; ++u) g->row_ptr[u + 1] += g->row_ptr[u];
    free(keepmap);
    return g;
}

/* Undirected edge list -> cleaned CSR (both directions, no loops, no dups). */
gg_graph *gg_from_edges(int32_t n, int64_t ne, const int32_t *src, const int32_t *dst, int lcc)
{
    int sh = gg_bits(n);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * ne + 1));
    if (!keys) return NULL;
    int64_t len = 0;
    for (int64_t k = 0; k < ne; ++k) {
        uint64_t a = (uint64_t)(uint32_t)src[k], b = (uint64_t)(uint32_t)dst[k];
        if (a == b || a >= (uint64_t)n || b >= (uint64_t)n) continue;
        keys[len++] = (a << sh) | b;
        keys[len++] = (b << sh) | a;
    }
    if (gg_radix(keys, len, 2 * sh) != 0) { free(keys); return NULL; }
    int64_t u = 0;
    for (int64_t k = 0; k < len; ++k)
        if (k == 0 || keys[k] != keys[k - 1]) keys[u++] = keys[k];
    gg_graph *g = gg_keys_to_graph(n, keys, u, sh, lcc);
    free(keys);
    return g;
}

/* Erdos-Renyi G(n, p): every pair independently with probability p, drawn by
 * geometric skipping over the pairs (w < v) in lexicographic order. */
gg_graph *gg_er(int32_t n, double p, uint64_t seed, int lcc)
{
    gg_rng r = {seed * 0x2545F4914F6CDD1Dull + 1};
    int64_t cap = 1024, ne = 0;
    int32_t *s = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap), *t = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    if (p > 0.0) {
        double lq = log1p(-p);
        int64_t v = 1, w = -1;
        while (v < n) {
            double u = gg_unif(&r);
            w += 1 + (p >= 1.0 ? 0 : (int64_t)floor(log1p(-u) / lq));
            while (w >= v && v < n) { w -= v; v++; }
            if (v < n) {
                if (ne == cap) {
                    cap *= 2;
                    s = (int32_t *)realloc(s, sizeof(int32_t) * (size_t)cap);
                    t = (int32_t *)realloc(t, sizeof(int32_t) * (size_t)cap);
                }
                s[ne] = (int32_t)v; t[ne] = (int32_t)w; ne++;
            }
        }
    }
    gg_graph *g = gg_from_edges(n, ne, s, t, lcc);
    free(s); free(t);
    return g;
}

/* Barabasi-Albert: a clique on m+1 seed nodes, then every new node attaches
 * to m distinct existing nodes drawn with probability proportional to degree
 * (uniform draws from the list of edge endpoints; repeated targets redrawn). */
gg_graph *gg_ba(int32_t n, int32_t m, uint64_t seed)
{
    if (m < 1 || n < m + 2) return NULL;
    gg_rng r = {seed * 0x2545F4914F6CDD1Dull + 2};
    int64_t ne_max = (int64_t)m * (m + 1) / 2 + (int64_t)(n - m - 1) * m;
    int32_t *s = (int32_t *)malloc(sizeof(int32_t) * (size_t)ne_max);
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (size_t)ne_max);
    int32_t *ends = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * ne_max));
    int32_t *pick = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
    int64_t ne = 0, ln = 0;
    for (int32_t a = 0; a <= m; ++a)
        for (int32_t b = a + 1; b <= m; ++b) {
            s[ne] = a; t[ne] = b; ne++;
            ends[ln++] = a; ends[ln++] = b;
        }
    for (int32_t v = m + 1; v < n; ++v) {
        for (int32_t k = 0; k < m; ++k) {
            for (;;) {
                int32_t c = ends[gg_below(&r, (uint64_t)ln)];
                int dup = 0;
                for (int32_t q = 0; q < k; ++q) if (pick[q] == c) { dup = 1; break; }
                if (!dup) { pick[k] = c; break; }
            }
        }
        for (int32_t k = 0; k < m; ++k) {
            s[ne] = v; t[ne] = pick[k]; ne++;
            ends[ln++] = v; ends[ln++] = pick[k];
        }
    }
    gg_graph *g = gg_from_edges(n, ne, s, t, 0);
    free(s); free(t); free(ends); free(pick);
    return g;
}

/* R-MAT (Chakrabarti, Zhan, Faloutsos 2004): each of n_edges edges descends
 * `scale` levels of the adjacency matrix, picking quadrant (0,0), (0,1), (1,0),
 * (1,1) with probabilities a, b, c, 1-a-b-c.  No noise. */
gg_graph *gg_rmat(int32_t scale, int64_t n_edges, double a, double b, double c, uint64_t seed, int lcc)
{
    int32_t n = (int32_t)1 << scale;
    gg_rng r = {seed * 0x2545F4914F6CDD1Dull + 3};
    int32_t *s = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_edges > 0 ? n_edges : 1));
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_edges > 0 ? n_edges : 1));
    if (!s || !t) { free(s); free(t); return NULL; }
    double ab = a + b, abc = a + b + c;
    for (int64_t e = 0; e < n_edges; ++e) {
        int32_t u = 0, w = 0;
        for (int32_t l = 0; l < scale; ++l) {
            double x = gg_unif(&r);
            int bu = x >= ab, bw = (x >= a && x < ab) || x >= abc;
            u = (u << 1) | bu;
            w = (w << 1) | bw;
        }
        s[e] = u; t[e] = w;
    }
    gg_graph *g = gg_from_edges(n, n_edges, s, t, lcc);
    free(s); free(t);
    return g;
}

void gg_free(gg_graph *g)
{
    if (!g) return;
    free(g->row_ptr); free(g->col); free(g->orig_id); free(g);
}
