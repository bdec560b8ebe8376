// FP64 solves with L_v (the Laplacian without row and column v, Section 3.1)
// on the GPU: conjugate gradients (Hestenes and Stiefel, 1952) with the
// Jacobi preconditioner D^{-1}.  L_v is symmetric positive definite for a
// connected graph.  The quantities the samplers estimate that are linear in
// L_v^{-1} applied to a known vector come out exactly (to the tolerance):
// L_v^{-1} 1 gives y2 (Alg. 2) and the row-sum terms of (L^+)_uu (Section
// 3.1, element-wise Theorem 1); L_v^{-1} d gives the hitting times h(., v)
// and E[Y2] (Section 3.2, Alg. 4).
//
// All reductions have a fixed order (per-chunk block sums, then one block),
// so the iterates are the same run to run.
#include "lap_internal.h"

namespace {

constexpr int kBlock = 256;
constexpr int kParts = 1024;

__device__ double block_sum(double x)
{
    __shared__ double sh[kBlock];
    sh[threadIdx.x] = x;
    __syncthreads();
    for (int w = kBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] = __dadd_rn(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

int grid_for(int64_t work)
{
    int64_t g = (work + kBlock - 1) / kBlock;
    return (int)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

#define NODE_LOOP(u, n) for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < (n); u += (int64_t)gridDim.x * blockDim.x)

// y = L_v x (x[v] read as 0, y[v] = 0): y_u = d_u x_u - sum_{w in N(u), w != v} x_w.
__global__ void lv_matvec(const int2 *__restrict__ rowinfo, const int32_t *__restrict__ col, int32_t n, int32_t v,
                          const double *__restrict__ x, double *__restrict__ y)
{
    NODE_LOOP(u, n)
    {
        if (u == v) { y[u] = 0.0; continue; }
        const int2 r = rowinfo[u];
        double a = 0.0;
        for (int32_t e = 0; e < r.y; ++e) {
            const int32_t w = col[(int64_t)r.x + e];
            if (w != v) a = __dadd_rn(a, x[w]);
        }
        y[u] = __dsub_rn(__dmul_rn((double)r.y, x[u]), a);
    }
}

// Partial sums of a[u] * b[u] over chunk p of the nodes.
__global__ void dot_partial(int32_t n, const double *__restrict__ a, const double *__restrict__ b, int64_t chunk,
                            double *__restrict__ part)
{
    const int64_t lo = (int64_t)blockIdx.x * chunk;
    const int64_t hi = lo + chunk < n ? lo + chunk : n;
    double acc = 0.0;
    for (int64_t u = lo + threadIdx.x; u < hi; u += kBlock) acc = __dadd_rn(acc, __dmul_rn(a[u], b[u]));
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void total_kernel(const double *__restrict__ part, double *out)
{
    double acc = 0.0;
    for (int k = threadIdx.x; k < kParts; k += kBlock) acc = __dadd_rn(acc, part[k]);
    acc = block_sum(acc);
    if (threadIdx.x == 0) *out = acc;
}

// r = b (b[v] = 0), z = r / d, p = z, x = 0.
__global__ void cg_init(const int2 *__restrict__ rowinfo, int32_t n, int32_t v, const double *__restrict__ b,
                        double *x, double *r, double *z, double *p)
{
    NODE_LOOP(u, n)
    {
        const double bu = (u == v) ? 0.0 : b[u];
        x[u] = 0.0;
        r[u] = bu;
        const double zu = __ddiv_rn(bu, (double)rowinfo[u].y);
        z[u] = zu;
        p[u] = zu;
    }
}

// x += alpha p, r -= alpha q, z = r / d (alpha = s[0] / s[1]).
__global__ void cg_update(const int2 *__restrict__ rowinfo, int32_t n, const double *s, const double *__restrict__ p,
                          const double *__restrict__ q, double *x, double *r, double *z)
{
    const double alpha = __ddiv_rn(s[0], s[1]);
    NODE_LOOP(u, n)
    {
        x[u] = __fma_rn(alpha, p[u], x[u]);
        const double ru = __fma_rn(-alpha, q[u], r[u]);
        r[u] = ru;
        z[u] = __ddiv_rn(ru, (double)rowinfo[u].y);
    }
}

// p = z + beta p (beta = s_new / s_old).
__global__ void cg_direction(int32_t n, const double *s_new, const double *s_old, const double *__restrict__ z, double *p)
{
    const double beta = __ddiv_rn(*s_new, *s_old);
    NODE_LOOP(u, n) p[u] = __fma_rn(beta, p[u], z[u]);
}

}  // namespace

// Solves L_v x = b on the device.  scratch: 4 n + 2 kParts + 8 doubles.
// Host-side loop: one scalar read per iteration (the residual norm).
cudaError_t lap_run_lv_solve(const int2 *rowinfo, const int32_t *col, int32_t n, int32_t v, const double *b, double *x,
                             double *scratch, double rtol, int32_t maxiter, int32_t *iterations, double *residual,
                             cudaStream_t st)
{
    double *r = scratch, *z = r + n, *p = z + n, *q = p + n, *part = q + n, *s = part + kParts;
    // s[0] = r.z, s[1] = p.q, s[2] = r.r, s[3] = b.b, s[4] = the next r.z
    const int64_t chunk = ((int64_t)n + kParts - 1) / kParts;
    const int grid = grid_for(n);
    cg_init<<<grid, kBlock, 0, st>>>(rowinfo, n, v, b, x, r, z, p);
    dot_partial<<<kParts, kBlock, 0, st>>>(n, r, z, chunk, part);
    total_kernel<<<1, kBlock, 0, st>>>(part, s + 0);
    dot_partial<<<kParts, kBlock, 0, st>>>(n, r, r, chunk, part);
    total_kernel<<<1, kBlock, 0, st>>>(part, s + 3);
    double h[5] = {0, 0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(h, s, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    const double bnorm = sqrt(h[3]);
    *iterations = 0;
    *residual = 0.0;
    if (bnorm == 0.0) return cudaMemsetAsync(x, 0, sizeof(double) * (size_t)n, st);
    for (int32_t it = 1; it <= maxiter; ++it) {
        lv_matvec<<<grid, kBlock, 0, st>>>(rowinfo, col, n, v, p, q);
        dot_partial<<<kParts, kBlock, 0, st>>>(n, p, q, chunk, part);
        total_kernel<<<1, kBlock, 0, st>>>(part, s + 1);
        cg_update<<<grid, kBlock, 0, st>>>(rowinfo, n, s, p, q, x, r, z);
        dot_partial<<<kParts, kBlock, 0, st>>>(n, r, r, chunk, part);
        total_kernel<<<1, kBlock, 0, st>>>(part, s + 2);
        dot_partial<<<kParts, kBlock, 0, st>>>(n, r, z, chunk, part);
        total_kernel<<<1, kBlock, 0, st>>>(part, s + 4);
        e = cudaMemcpyAsync(h, s, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        *iterations = it;
        *residual = sqrt(h[2]) / bnorm;
        if (*residual <= rtol) break;
        cg_direction<<<grid, kBlock, 0, st>>>(n, s + 4, s + 0, z, p);
        e = cudaMemcpyAsync(s + 0, s + 4, sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}
