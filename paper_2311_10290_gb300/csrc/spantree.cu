// SpanTree estimators (Alg. 1 for ECC, Alg. 3 for Kemeny's constant).
//
// Section 4.1: the electrical flow of G is the average of the flows sent on
// its uniform spanning trees, so a voltage of G (the sum of edge flows along
// a fixed path to the landmark v) is the average over trees of the same sum
// of tree flows.  With a fixed BFS tree from v (parent of u: its smallest-id
// neighbour one hop closer to v), a sampled tree T (parent array next[]) adds
// for every node u and every edge (e1 -> e2 = bfs_parent(e1)) of u's BFS path:
//   x1(u)  += 1 if next[e1] == e2 and u is in T's subtree of e1,
//             -1 if next[e2] == e1 and u is in T's subtree of e2
//             (unit current from u to v flows on T's path from u only);
//   x2(u)  += |subtree(e1)| if next[e1] == e2,  -|subtree(e2)| if next[e2] == e1
//             (1/n injected at every node: the tree edge (a, next[a]) carries
//             |subtree(a)| / n whatever u is);
//   x2d(u) += the same with subtree degree sums (d_w / 2m injected at w, Alg. 3).
// E[x1(u)] = (L_v^{-1})_uu, E[x2(u)] / n = (1/n) e_u^T L_v^{-1} 1,
// E[sum_u d_u x1(u)] = Tr((I - P_v)^{-1}), E[sum_u d_u x2d(u)] / 2m = (1/2m) d^T L_v^{-1} d.
// (Alg. 1 prints the subtree test the other way round and applies it to x2
// as well; the text and the flow argument fix the reading used here.)
//
// The trees come from the 8-byte Wilson kernel run with one sample per lane
// (its slot ends holding Next of every node).  One CTA processes one tree:
// children lists by counting sort, the tree's levels from v, subtree sizes
// and degree sums bottom-up, preorder intervals top-down, then the BFS-path
// sums for every node.  All per-node sums are integers, so accumulating them
// over trees with atomics is exact and deterministic.
#include "lap_internal.h"

namespace {

constexpr int kTB = 512;          // threads per tree CTA
constexpr int kFB = 256;          // finalize block
constexpr int kParts = 1024;      // finalize partial sums (fixed order)

__device__ __forceinline__ int32_t parent_of(const unsigned long long *tree, int32_t u)
{
    return (int32_t)(uint32_t)tree[u];
}

// Exclusive prefix sum of in[0..n) into out[0..n] (out[n] = total), by one CTA.
__device__ void block_exclusive_scan(const int32_t *in, int32_t *out, int32_t n)
{
    __shared__ int32_t warp_tot[kTB / 32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int32_t base = 0; base < n; base += kTB) {
        const int32_t idx = base + (int32_t)threadIdx.x;
        const int32_t x = idx < n ? in[idx] : 0;
        int32_t incl = x;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int32_t t = lane < kTB / 32 ? warp_tot[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
                if (lane >= o) t += y;
            }
            if (lane < kTB / 32) warp_tot[lane] = t;     // inclusive over warps
        }
        __syncthreads();
        const int32_t before = carry + (wid ? warp_tot[wid - 1] : 0);
        if (idx < n) out[idx] = before + incl - x;
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_tot[kTB / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry;
    __syncthreads();
}

__global__ void bfs_parent_kernel(const int2 *__restrict__ rowinfo, const int32_t *__restrict__ col,
                                  const int32_t *__restrict__ hops, int32_t n, int32_t root, int32_t *bpar,
                                  unsigned int *status)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        if (u == root) { bpar[u] = -1; continue; }
        const int2 r = rowinfo[u];
        const int32_t want = hops[u] - 1;
        int32_t best = -1;
        for (int32_t e = 0; e < r.y; ++e) {
            const int32_t w = col[r.x + e];
            if (hops[w] == want && (best < 0 || w < best)) best = w;
        }
        bpar[u] = best;
        if (best < 0) atomicOr(status, LAP_DEV_BAD_INDEX);
    }
}

__global__ void __launch_bounds__(kTB) spantree_tree_kernel(LapSpanTreeLaunch p)
{
    const int32_t n = p.n, v = p.root;
    long long *dsum = reinterpret_cast<long long *>(p.scratch + (uint64_t)blockIdx.x * p.scratch_ints);
    int32_t *cnt = reinterpret_cast<int32_t *>(dsum + n);
    int32_t *off = cnt + n;             // n + 1
    int32_t *child = off + n + 1;       // n
    int32_t *queue = child + n;         // n
    int32_t *lstart = queue + n;        // n + 2
    int32_t *size = lstart + n + 2;     // n
    int32_t *pre = size + n;            // n
    __shared__ int32_t tail;
    __shared__ int32_t levels;
    const int32_t tid = (int32_t)threadIdx.x;

    for (uint32_t j = blockIdx.x; j < p.count; j += gridDim.x) {
        const unsigned long long *T = p.trees + (uint64_t)j * (uint64_t)n;
        // Children lists of T (counting sort by parent).
        for (int32_t u = tid; u < n; u += kTB) {
            cnt[u] = 0;
            size[u] = 1;
            dsum[u] = p.rowinfo[u].y;
        }
        __syncthreads();
        for (int32_t u = tid; u < n; u += kTB) {
            if (u == v) continue;
            const int32_t a = parent_of(T, u);
            if ((uint32_t)a >= (uint32_t)n) { atomicOr(p.status, LAP_DEV_BAD_INDEX); continue; }
            atomicAdd(&cnt[a], 1);
        }
        __syncthreads();
        block_exclusive_scan(cnt, off, n);
        for (int32_t u = tid; u < n; u += kTB) cnt[u] = 0;
        __syncthreads();
        for (int32_t u = tid; u < n; u += kTB) {
            if (u == v) continue;
            const int32_t a = parent_of(T, u);
            if ((uint32_t)a >= (uint32_t)n) continue;
            child[off[a] + atomicAdd(&cnt[a], 1)] = u;
        }
        __syncthreads();
        // Levels of T from v (queue holds the nodes level by level).
        if (tid == 0) {
            queue[0] = v;
            lstart[0] = 0;
            lstart[1] = 1;
            tail = 1;
            levels = 1;
        }
        __syncthreads();
        for (int32_t L = 0;; ++L) {
            const int32_t a = lstart[L], b = lstart[L + 1];
            if (a == b || b >= n) break;
            for (int32_t idx = a + tid; idx < b; idx += kTB) {
                const int32_t u = queue[idx];
                for (int32_t c = off[u]; c < off[u + 1]; ++c) {
                    const int32_t pos = atomicAdd(&tail, 1);
                    if (pos < n) queue[pos] = child[c];
                }
            }
            __syncthreads();
            if (tid == 0) {
                lstart[L + 2] = tail < n ? tail : n;
                levels = L + 2;
            }
            __syncthreads();
        }
        if (tid == 0 && tail != n) atomicOr(p.status, LAP_DEV_BAD_INDEX);   // not a spanning tree
        __syncthreads();
        const int32_t nl = levels;       // levels 0 .. nl-1 hold nodes
        // Subtree sizes and degree sums, deepest level first.
        for (int32_t L = nl - 1; L >= 1; --L) {
            for (int32_t idx = lstart[L] + tid; idx < lstart[L + 1]; idx += kTB) {
                const int32_t u = queue[idx];
                const int32_t a = parent_of(T, u);
                atomicAdd(&size[a], size[u]);
                atomicAdd(reinterpret_cast<unsigned long long *>(&dsum[a]), (unsigned long long)dsum[u]);
            }
            __syncthreads();
        }
        // Preorder intervals: u's subtree is [pre[u], pre[u] + size[u]).
        if (tid == 0) pre[v] = 0;
        __syncthreads();
        for (int32_t L = 0; L < nl - 1; ++L) {
            for (int32_t idx = lstart[L] + tid; idx < lstart[L + 1]; idx += kTB) {
                const int32_t u = queue[idx];
                int32_t next_pre = pre[u] + 1;
                for (int32_t c = off[u]; c < off[u + 1]; ++c) {
                    const int32_t w = child[c];
                    pre[w] = next_pre;
                    next_pre += size[w];
                }
            }
            __syncthreads();
        }
        // The sums along every node's BFS path.
        for (int32_t u = tid; u < n; u += kTB) {
            long long x1 = 0, x2 = 0, x2d = 0;
            const int32_t pu = pre[u];
            int32_t e1 = u;
            for (int32_t guard = 0; e1 != v && guard < n; ++guard) {
                const int32_t e2 = p.bpar[e1];
                if ((uint32_t)e2 >= (uint32_t)n) { atomicOr(p.status, LAP_DEV_BAD_INDEX); break; }
                if (parent_of(T, e1) == e2) {
                    x2 += size[e1];
                    x2d += dsum[e1];
                    if (pre[e1] <= pu && pu < pre[e1] + size[e1]) ++x1;
                } else if (e2 != v && parent_of(T, e2) == e1) {
                    x2 -= size[e2];
                    x2d -= dsum[e2];
                    if (pre[e2] <= pu && pu < pre[e2] + size[e2]) --x1;
                }
                e1 = e2;
            }
            if (x1) atomicAdd(&p.x1[u], (unsigned long long)x1);
            if (x2) atomicAdd(&p.x2[u], (unsigned long long)x2);
            if (x2d) atomicAdd(&p.x2d[u], (unsigned long long)x2d);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ finalize

__device__ double fblock_sum(double x)
{
    __shared__ double sh[kFB];
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int w = kFB / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// which 0: sum x2(u) = X2[u] / (n omega); 1: sum ldiag; 2: sum d_u X1[u]; 3: sum d_u X2d[u].
__global__ void st_partial_kernel(const int2 *__restrict__ rowinfo, int32_t n, double omega,
                                  const long long *__restrict__ X1, const long long *__restrict__ X2,
                                  const long long *__restrict__ X2d, const double *__restrict__ ldiag, int which,
                                  double *part)
{
    const int64_t chunk = ((int64_t)n + kParts - 1) / kParts;
    const int64_t a = (int64_t)blockIdx.x * chunk;
    const int64_t b = a + chunk < n ? a + chunk : n;
    const double nw = __dmul_rn((double)n, omega);
    double acc = 0.0;
    for (int64_t u = a + threadIdx.x; u < b; u += kFB) {
        double x;
        if (which == 0) x = __ddiv_rn((double)X2[u], nw);
        else if (which == 1) x = ldiag[u];
        else if (which == 2) x = (double)((long long)rowinfo[u].y * X1[u]);
        else x = (double)((long long)rowinfo[u].y * X2d[u]);
        acc = __dadd_rn(acc, x);
    }
    acc = fblock_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void st_total_kernel(const double *part, double *out)
{
    double acc = 0.0;
    for (int k = threadIdx.x; k < kParts; k += kFB) acc = __dadd_rn(acc, part[k]);
    acc = fblock_sum(acc);
    if (threadIdx.x == 0) *out = acc;
}

__global__ void st_ldiag_kernel(int32_t n, int32_t root, double omega, const long long *__restrict__ X1,
                                const long long *__restrict__ X2, const double *s2, double *ldiag)
{
    const double mean = __ddiv_rn(*s2, (double)n);
    const double nw = __dmul_rn((double)n, omega);
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        if (u == root) { ldiag[u] = mean; continue; }
        const double x1 = __ddiv_rn((double)X1[u], omega);
        const double x2 = __ddiv_rn((double)X2[u], nw);
        ldiag[u] = __dadd_rn(__dsub_rn(x1, __dmul_rn(2.0, x2)), mean);
    }
}

__global__ void st_ecc_kernel(int32_t n, const double *__restrict__ ldiag, const double *tr, double *ecc)
{
    const double t = *tr;
    const double num = (double)(n - 1);
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        ecc[u] = __ddiv_rn(num, __dadd_rn(__dmul_rn((double)n, ldiag[u]), t));
}

int fgrid(int64_t n)
{
    int64_t g = (n + kFB - 1) / kFB;
    return (int)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

}  // namespace

cudaError_t lap_launch_bfs_parent(const int2 *rowinfo, const int32_t *col, const int32_t *hops, int32_t n, int32_t root,
                                  int32_t *bpar, unsigned int *status, cudaStream_t st)
{
    bfs_parent_kernel<<<fgrid(n), kFB, 0, st>>>(rowinfo, col, hops, n, root, bpar, status);
    return cudaGetLastError();
}

uint64_t lap_spantree_scratch_ints(int32_t n)
{
    // dsum (2n ints) + cnt n + off n+1 + child n + queue n + lstart n+2 + size n + pre n, rounded to even.
    const uint64_t ints = 2ull * (uint64_t)n + 7ull * (uint64_t)n + 3ull;
    return (ints + 1ull) & ~1ull;
}

int lap_spantree_block() { return kTB; }

cudaError_t lap_launch_spantree(const LapSpanTreeLaunch &p, int blocks, cudaStream_t st)
{
    if (p.count == 0 || blocks <= 0) return cudaSuccess;
    spantree_tree_kernel<<<blocks, kTB, 0, st>>>(p);
    return cudaGetLastError();
}

// red: kParts + 4 doubles (partials, then sum x2, trace, sum d X1, sum d X2d).
cudaError_t lap_launch_spantree_finalize(const int2 *rowinfo, int32_t n, int32_t root, uint64_t omega,
                                         const long long *X1, const long long *X2, const long long *X2d,
                                         double *ldiag, double *ecc, double *red, cudaStream_t st)
{
    const double w = (double)omega;
    double *part = red;
    st_partial_kernel<<<kParts, kFB, 0, st>>>(rowinfo, n, w, X1, X2, X2d, nullptr, 0, part);
    st_total_kernel<<<1, kFB, 0, st>>>(part, red + kParts);
    st_ldiag_kernel<<<fgrid(n), kFB, 0, st>>>(n, root, w, X1, X2, red + kParts, ldiag);
    st_partial_kernel<<<kParts, kFB, 0, st>>>(rowinfo, n, w, X1, X2, X2d, ldiag, 1, part);
    st_total_kernel<<<1, kFB, 0, st>>>(part, red + kParts + 1);
    st_ecc_kernel<<<fgrid(n), kFB, 0, st>>>(n, ldiag, red + kParts + 1, ecc);
    st_partial_kernel<<<kParts, kFB, 0, st>>>(rowinfo, n, w, X1, X2, X2d, nullptr, 2, part);
    st_total_kernel<<<1, kFB, 0, st>>>(part, red + kParts + 2);
    st_partial_kernel<<<kParts, kFB, 0, st>>>(rowinfo, n, w, X1, X2, X2d, nullptr, 3, part);
    st_total_kernel<<<1, kFB, 0, st>>>(part, red + kParts + 3);
    return cudaGetLastError();
}
