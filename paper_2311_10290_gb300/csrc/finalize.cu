// FP64 finalize (hot-path row a6): integer counts -> (L^+)_uu, ECC, Kemeny.
//
//   y1(u) = cnt1[u] / (omega d_u)    estimates (L_v^{-1})_uu          (Alg. 2; LE-walk lemma)
//   y2(u) = cnt2[u] / (omega d_u)    estimates (1/n) e_u^T L_v^{-1} 1 (Alg. 2; "sample the paths")
//   (L^+)_uu = y1(u) - 2 y2(u) + (1/n) sum_w y2(w)   (u != v; element-wise Thm 1)
//   (L^+)_vv = (1/n) sum_w y2(w)
//   c(u) = (n-1) / (n (L^+)_uu + sum_w (L^+)_ww)     (Section 2, ECC)
// with cnt1[u] = omega + (repeat visits of u) for u != v.
//
// Sums use a fixed two-level order (per-block tree, then one block over the
// partials), so results are deterministic run to run.  All arithmetic uses
// explicitly rounded operations (no FMA contraction).
#include "lap_internal.h"

namespace {

constexpr int kBlock = 256;
constexpr int kParts = 1024;   // number of partial sums (fixed)

__device__ __forceinline__ double y_of(unsigned long long c, double wd) { return __ddiv_rn((double)c, wd); }

__device__ double block_sum(double x)
{
    __shared__ double sh[kBlock];
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// Partial p covers nodes [p*chunk, (p+1)*chunk).  which = 0: sum of y2;
// which = 1: sum of ldiag.
__global__ void partial_kernel(const int2 *__restrict__ rowinfo, int32_t n, double omega,
                               const unsigned long long *__restrict__ cnt2, const double *__restrict__ ldiag,
                               int which, int64_t chunk, double *part)
{
    const int64_t a = (int64_t)blockIdx.x * chunk;
    const int64_t b = a + chunk < n ? a + chunk : n;
    double acc = 0.0;
    for (int64_t u = a + threadIdx.x; u < b; u += kBlock) {
        double x;
        if (which == 0) x = y_of(cnt2[u], __dmul_rn(omega, (double)rowinfo[u].y));
        else x = ldiag[u];
        acc = __dadd_rn(acc, x);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void total_kernel(const double *part, int parts, double *out)
{
    double acc = 0.0;
    for (int k = threadIdx.x; k < parts; k += kBlock) acc = __dadd_rn(acc, part[k]);
    acc = block_sum(acc);
    if (threadIdx.x == 0) *out = acc;
}

__global__ void ldiag_kernel(const int2 *__restrict__ rowinfo, int32_t n, int32_t root, double omega,
                             unsigned long long omega_u, const unsigned long long *__restrict__ rep1,
                             const unsigned long long *__restrict__ cnt2, const double *s2, double *ldiag)
{
    const double lvv = __ddiv_rn(*s2, (double)n);
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        if (u == root) { ldiag[u] = lvv; continue; }
        const double wd = __dmul_rn(omega, (double)rowinfo[u].y);
        const double y1 = y_of(omega_u + rep1[u], wd);
        const double y2 = y_of(cnt2[u], wd);
        ldiag[u] = __dadd_rn(__dsub_rn(y1, __dmul_rn(2.0, y2)), lvv);
    }
}

__global__ void ecc_kernel(int32_t n, const double *__restrict__ ldiag, const double *tr, double *ecc)
{
    const double t = *tr;
    const double num = (double)(n - 1);
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        ecc[u] = __ddiv_rn(num, __dadd_rn(__dmul_rn((double)n, ldiag[u]), t));
}

// Random-walk betweenness (Section 5, "Discussions"):
//   c_b(u) = 1/n + Tr(L^+) / ((n-1) (Tr(L^+) + n (L^+)_uu)).
__global__ void rwb_kernel(int32_t n, const double *__restrict__ ldiag, const double *tr, double *out)
{
    const double t = *tr;
    const double inv_n = __ddiv_rn(1.0, (double)n);
    const double nm1 = (double)(n - 1);
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        out[u] = __dadd_rn(inv_n, __ddiv_rn(t, __dmul_rn(nm1, __dadd_rn(t, __dmul_rn((double)n, ldiag[u])))));
}

// out[u] = cnt2[u] / (omega d_u): with the first absorbed walk started at a
// fixed s, the passes of u have mean d_u (L_v^{-1})_{su} (Section 4.2,
// "v-absorbed walk" lemma), so this is row s of L_v^{-1}; with the uniform
// start it is y2(u) of Alg. 2.
__global__ void lv_row_kernel(const int2 *__restrict__ rowinfo, int32_t n, double omega,
                              const unsigned long long *__restrict__ cnt2, double *out)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        out[u] = y_of(cnt2[u], __dmul_rn(omega, (double)rowinfo[u].y));
}

__global__ void counts_kernel(int32_t n, int32_t root, unsigned long long omega,
                              const unsigned long long *__restrict__ rep1, unsigned long long *cnt1)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        cnt1[u] = (u == root) ? 0ull : omega + rep1[u];
}

// Batched forms: blockIdx.y is the graph; per graph the same chunks, block
// reductions and operation order as the single-graph kernels above, so each
// graph's results are bit-identical to lap_launch_finalize on that graph.
constexpr int kRedStride = kParts + 2;

__global__ void partial_batch_kernel(const LapBatchGraph *__restrict__ gs, double omega, int which, double *red)
{
    const LapBatchGraph &g = gs[blockIdx.y];
    const int32_t n = g.n;
    const int64_t chunk = ((int64_t)n + kParts - 1) / kParts;
    const int64_t a = (int64_t)blockIdx.x * chunk;
    const int64_t b = a + chunk < n ? a + chunk : n;
    double acc = 0.0;
    for (int64_t u = a + threadIdx.x; u < b; u += kBlock) {
        double x;
        if (which == 0) x = y_of(g.cnt2[u], __dmul_rn(omega, (double)g.rowinfo[u].y));
        else x = g.ldiag[u];
        acc = __dadd_rn(acc, x);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) red[(int64_t)blockIdx.y * kRedStride + blockIdx.x] = acc;
}

__global__ void total_batch_kernel(int which, double *red)
{
    double *part = red + (int64_t)blockIdx.x * kRedStride;
    double acc = 0.0;
    for (int k = threadIdx.x; k < kParts; k += kBlock) acc = __dadd_rn(acc, part[k]);
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[kParts + which] = acc;
}

__global__ void ldiag_batch_kernel(const LapBatchGraph *__restrict__ gs, double omega, unsigned long long omega_u,
                                   const double *red)
{
    const LapBatchGraph &g = gs[blockIdx.y];
    const int32_t n = g.n;
    const double lvv = __ddiv_rn(red[(int64_t)blockIdx.y * kRedStride + kParts], (double)n);
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        if (u == g.root) { g.ldiag[u] = lvv; continue; }
        const double wd = __dmul_rn(omega, (double)g.rowinfo[u].y);
        const double y1 = y_of(omega_u + g.rep1[u], wd);
        const double y2 = y_of(g.cnt2[u], wd);
        g.ldiag[u] = __dadd_rn(__dsub_rn(y1, __dmul_rn(2.0, y2)), lvv);
    }
}

__global__ void ecc_batch_kernel(const LapBatchGraph *__restrict__ gs, const double *red)
{
    const LapBatchGraph &g = gs[blockIdx.y];
    const int32_t n = g.n;
    const double t = red[(int64_t)blockIdx.y * kRedStride + kParts + 1];
    const double num = (double)(n - 1);
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        g.ecc[u] = __ddiv_rn(num, __dadd_rn(__dmul_rn((double)n, g.ldiag[u]), t));
}

// rep1[u] = cnt1[u] - omega (u != v); flags counts that cannot come from
// omega samples (cnt1[v] != 0 or cnt1[u] < omega).
__global__ void rep_from_counts_kernel(int32_t n, int32_t root, unsigned long long omega,
                                       const unsigned long long *__restrict__ cnt1, unsigned long long *rep1,
                                       unsigned int *bad)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long c = cnt1[u];
        if (u == root) {
            rep1[u] = 0ull;
            if (c != 0ull) atomicOr(bad, 1u);
        } else {
            rep1[u] = c >= omega ? c - omega : 0ull;
            if (c < omega) atomicOr(bad, 1u);
        }
    }
}

int grid_for(int64_t n)
{
    int64_t g = (n + kBlock - 1) / kBlock;
    return (int)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

}  // namespace

// red must hold kParts + 2 doubles: partials, then sum y2, then trace.
cudaError_t lap_launch_finalize(const int2 *rowinfo, int32_t n, int32_t root, uint64_t omega,
                                const unsigned long long *rep1, const unsigned long long *cnt2,
                                double *ldiag, double *ecc, double *red, cudaStream_t st)
{
    const double w = (double)omega;
    const int64_t chunk = ((int64_t)n + kParts - 1) / kParts;
    double *part = red, *s2 = red + kParts, *tr = red + kParts + 1;
    partial_kernel<<<kParts, kBlock, 0, st>>>(rowinfo, n, w, cnt2, nullptr, 0, chunk, part);
    total_kernel<<<1, kBlock, 0, st>>>(part, kParts, s2);
    ldiag_kernel<<<grid_for(n), kBlock, 0, st>>>(rowinfo, n, root, w, (unsigned long long)omega, rep1, cnt2, s2, ldiag);
    partial_kernel<<<kParts, kBlock, 0, st>>>(rowinfo, n, w, nullptr, ldiag, 1, chunk, part);
    total_kernel<<<1, kBlock, 0, st>>>(part, kParts, tr);
    ecc_kernel<<<grid_for(n), kBlock, 0, st>>>(n, ldiag, tr, ecc);
    return cudaGetLastError();
}

cudaError_t lap_launch_counts(int32_t n, int32_t root, uint64_t omega, const unsigned long long *rep1,
                              unsigned long long *cnt1, cudaStream_t st)
{
    counts_kernel<<<grid_for(n), kBlock, 0, st>>>(n, root, (unsigned long long)omega, rep1, cnt1);
    return cudaGetLastError();
}

cudaError_t lap_launch_finalize_batch(const LapBatchGraph *graphs, int32_t n_graphs, int32_t max_n, uint64_t omega,
                                      double *red, cudaStream_t st)
{
    if (n_graphs <= 0) return cudaSuccess;
    const double w = (double)omega;
    int gx = (int)(((int64_t)max_n + kBlock - 1) / kBlock);
    if (gx > 64) gx = 64;
    if (gx < 1) gx = 1;
    const dim3 parts(kParts, (unsigned)n_graphs), nodes((unsigned)gx, (unsigned)n_graphs);
    partial_batch_kernel<<<parts, kBlock, 0, st>>>(graphs, w, 0, red);
    total_batch_kernel<<<n_graphs, kBlock, 0, st>>>(0, red);
    ldiag_batch_kernel<<<nodes, kBlock, 0, st>>>(graphs, w, (unsigned long long)omega, red);
    partial_batch_kernel<<<parts, kBlock, 0, st>>>(graphs, w, 1, red);
    total_batch_kernel<<<n_graphs, kBlock, 0, st>>>(1, red);
    ecc_batch_kernel<<<nodes, kBlock, 0, st>>>(graphs, red);
    return cudaGetLastError();
}

cudaError_t lap_launch_rep_from_counts(int32_t n, int32_t root, uint64_t omega, const unsigned long long *cnt1,
                                       unsigned long long *rep1, unsigned int *bad, cudaStream_t st)
{
    rep_from_counts_kernel<<<grid_for(n), kBlock, 0, st>>>(n, root, (unsigned long long)omega, cnt1, rep1, bad);
    return cudaGetLastError();
}

// red as filled by lap_launch_finalize (trace at red[1024 + 1]).
cudaError_t lap_launch_rw_betweenness(int32_t n, const double *ldiag, const double *red, double *out, cudaStream_t st)
{
    rwb_kernel<<<grid_for(n), kBlock, 0, st>>>(n, ldiag, red + kParts + 1, out);
    return cudaGetLastError();
}

cudaError_t lap_launch_lv_row(const int2 *rowinfo, int32_t n, uint64_t omega, const unsigned long long *cnt2,
                              double *out, cudaStream_t st)
{
    lv_row_kernel<<<grid_for(n), kBlock, 0, st>>>(rowinfo, n, (double)omega, cnt2, out);
    return cudaGetLastError();
}
