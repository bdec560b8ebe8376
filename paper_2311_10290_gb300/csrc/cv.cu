// Control-variate support kernels (the paper has no control variate; see
// include/lap.h, lap_features .. lap_cv_estimates):
//   * 8 local node features for the MLP,
//   * integer potentials h = round(2^20 phi) and neighbour sums S[u],
//   * hitting-time targets: v-absorbed walks from every node (Section 3.2,
//     v-absorbed walk lemma: E[length from u] = h(u, v) = (L_v^{-1} d)_u),
//   * the CV finalize: Z1[u] = d_u A1[u] - cnt1[u] S1[u] and
//     M2 = sum_u (d_u A2[u] - P2[u] S2[u]) / d_u, then
//     y1_cv(u) = (cnt1[u] - beta1 Z1[u] / d_u) / (omega d_u) and
//     kappa_cv = (sum Y1 - sum Y2 + beta2 M2) / omega.
#include "lap_internal.h"
#include "philox.cuh"

namespace {

constexpr int kBlock = 256;
constexpr int kParts = 1024;

int grid_for(int64_t work)
{
    int64_t g = (work + kBlock - 1) / kBlock;
    return (int)(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

#define NODE_LOOP(u, n) for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < (n); u += (int64_t)gridDim.x * blockDim.x)

// s1[u] = sum of neighbour degrees, ones[u] = neighbours of degree 1.
__global__ void feat_pass1(const int2 *__restrict__ rowinfo, const int32_t *__restrict__ col, int32_t n,
                           double *__restrict__ s1, double *__restrict__ ones)
{
    NODE_LOOP(u, n)
    {
        const int2 r = rowinfo[u];
        double a = 0.0, b = 0.0;
        for (int32_t e = 0; e < r.y; ++e) {
            const int32_t d = rowinfo[col[r.x + e]].y;
            a += (double)d;
            b += d == 1 ? 1.0 : 0.0;
        }
        s1[u] = a;
        ones[u] = b;
    }
}

// out[u] = sum over neighbours x of in[x] (optionally divided by d_u, with
// out[v] = 1: one step of the "hit v within k steps" iteration).
__global__ void neighbour_sum_kernel(const int2 *__restrict__ rowinfo, const int32_t *__restrict__ col, int32_t n,
                                     const double *__restrict__ in, double *__restrict__ out, int32_t absorb_root)
{
    NODE_LOOP(u, n)
    {
        const int2 r = rowinfo[u];
        double a = 0.0;
        for (int32_t e = 0; e < r.y; ++e) a += in[col[r.x + e]];
        if (absorb_root >= 0) a = (u == absorb_root) ? 1.0 : a / (double)r.y;
        out[u] = a;
    }
}

__global__ void feat_assemble(const int2 *__restrict__ rowinfo, const int32_t *__restrict__ hops, int32_t n,
                              const double *__restrict__ s1, const double *__restrict__ s2,
                              const double *__restrict__ ones, const double *__restrict__ a, float *__restrict__ f)
{
    NODE_LOOP(u, n)
    {
        const double d = (double)rowinfo[u].y;
        float *o = f + u * 8;
        o[0] = (float)log(d);
        o[1] = (float)(1.0 / d);
        o[2] = (float)log1p((double)hops[u]);
        o[3] = hops[u] == 1 ? 1.f : 0.f;
        o[4] = (float)log(s1[u] / d);
        o[5] = (float)(ones[u] / d);
        o[6] = (float)log(s2[u] / s1[u]);
        o[7] = (float)a[u];
    }
}

__global__ void quantize_kernel(const double *__restrict__ phi, int32_t n, long long *__restrict__ h)
{
    NODE_LOOP(u, n) h[u] = __double2ll_rn(ldexp(phi[u], LAP_CV_FIXED_POINT_BITS));
}

__global__ void int_neighbour_sum_kernel(const int2 *__restrict__ rowinfo, const int32_t *__restrict__ col, int32_t n,
                                         const long long *__restrict__ h, long long *__restrict__ S)
{
    NODE_LOOP(u, n)
    {
        const int2 r = rowinfo[u];
        long long a = 0;
        for (int32_t e = 0; e < r.y; ++e) a += h[col[r.x + e]];
        S[u] = a;
    }
}

// One thread per (node, repetition): a walk from u absorbed at v; step t uses
// Philox counter (t, u, rep, 3).
__global__ void hitting_walks_kernel(LapDevGraph g, int32_t v, uint64_t seed, uint32_t reps, uint64_t limit,
                                     unsigned long long *__restrict__ sums, unsigned int *status)
{
    const uint64_t total = (uint64_t)g.n * reps;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (uint64_t pair = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; pair < total;
         pair += (uint64_t)gridDim.x * blockDim.x) {
        const int32_t u = (int32_t)(pair / reps);
        const uint32_t rep = (uint32_t)(pair % reps);
        uint64_t t = 0;
        int32_t x = u;
        bool bad = false;
        while (x != v) {
            ++t;
            if (t > limit) { bad = true; break; }
            const int2 r = g.rowinfo[x];
            x = g.col[r.x + (int64_t)lap::below(lap::philox_r64((uint32_t)t, (uint32_t)u, rep, 3u, k0, k1), (uint64_t)r.y)];
        }
        if (bad) atomicOr(status, (unsigned int)LAP_DEV_STEP_LIMIT);
        else if (t) atomicAdd(&sums[u], (unsigned long long)t);
    }
}

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

// Per-node CV terms.  which 0: Z1[u] (int64, written to z1); which 1:
// (d_u A2[u] - P2[u] S2[u]) / d_u partial sums.
__global__ void m2_partial_kernel(const int2 *__restrict__ rowinfo, int32_t n, const long long *__restrict__ a2,
                                  const long long *__restrict__ p2, const long long *__restrict__ S2, int64_t chunk,
                                  double *__restrict__ part)
{
    const int64_t a = (int64_t)blockIdx.x * chunk;
    const int64_t b = a + chunk < n ? a + chunk : n;
    double acc = 0.0;
    for (int64_t u = a + threadIdx.x; u < b; u += kBlock) {
        const long long d = rowinfo[u].y;
        const long long num = d * a2[u] - p2[u] * S2[u];
        acc = __dadd_rn(acc, __ddiv_rn((double)num, (double)d));
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

// Partial sums of y2 (plain) and of the CV diagonal, as in finalize.cu but
// with y1 replaced by the control-variate version.
__global__ void cv_y2_partial(const int2 *__restrict__ rowinfo, int32_t n, double omega,
                              const unsigned long long *__restrict__ cnt2, int64_t chunk, double *part)
{
    const int64_t a = (int64_t)blockIdx.x * chunk;
    const int64_t b = a + chunk < n ? a + chunk : n;
    double acc = 0.0;
    for (int64_t u = a + threadIdx.x; u < b; u += kBlock)
        acc = __dadd_rn(acc, __ddiv_rn((double)cnt2[u], __dmul_rn(omega, (double)rowinfo[u].y)));
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void cv_ldiag_kernel(const int2 *__restrict__ rowinfo, int32_t n, int32_t root, double omega,
                                unsigned long long omega_u, const unsigned long long *__restrict__ rep1,
                                const unsigned long long *__restrict__ cnt2, const long long *__restrict__ a1,
                                const long long *__restrict__ S1, double beta1, const double *s2, double *ldiag)
{
    const double lvv = __ddiv_rn(*s2, (double)n);
    NODE_LOOP(u, n)
    {
        if (u == root) { ldiag[u] = lvv; continue; }
        const long long d = rowinfo[u].y;
        const unsigned long long c1 = omega_u + rep1[u];
        const double wd = __dmul_rn(omega, (double)d);
        double cv = (double)c1;
        if (a1) {
            const long long z1 = d * a1[u] - (long long)c1 * S1[u];
            cv = __dsub_rn(cv, __dmul_rn(beta1, __ddiv_rn((double)z1, (double)d)));
        }
        const double y1 = __ddiv_rn(cv, wd);
        const double y2 = __ddiv_rn((double)cnt2[u], wd);
        ldiag[u] = __dadd_rn(__dsub_rn(y1, __dmul_rn(2.0, y2)), lvv);
    }
}

__global__ void ld_partial(int32_t n, const double *__restrict__ ld, int64_t chunk, double *part)
{
    const int64_t a = (int64_t)blockIdx.x * chunk;
    const int64_t b = a + chunk < n ? a + chunk : n;
    double acc = 0.0;
    for (int64_t u = a + threadIdx.x; u < b; u += kBlock) acc = __dadd_rn(acc, ld[u]);
    acc = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

__global__ void cv_ecc_kernel(int32_t n, const double *__restrict__ ldiag, const double *tr, double *ecc)
{
    const double t = *tr;
    const double num = (double)(n - 1);
    NODE_LOOP(u, n) ecc[u] = __ddiv_rn(num, __dadd_rn(__dmul_rn((double)n, ldiag[u]), t));
}

}  // namespace

cudaError_t lap_launch_features(const int2 *rowinfo, const int32_t *col, const int32_t *hops, int32_t n, int32_t root,
                                double *scratch /* 5 n */, float *feat, cudaStream_t st)
{
    double *s1 = scratch, *ones = scratch + n, *s2 = scratch + 2 * (int64_t)n, *a = scratch + 3 * (int64_t)n,
           *b = scratch + 4 * (int64_t)n;
    const int grid = grid_for(n);
    feat_pass1<<<grid, kBlock, 0, st>>>(rowinfo, col, n, s1, ones);
    neighbour_sum_kernel<<<grid, kBlock, 0, st>>>(rowinfo, col, n, s1, s2, -1);
    cudaError_t e = cudaMemsetAsync(a, 0, sizeof(double) * (size_t)n, st);
    if (e != cudaSuccess) return e;
    const double one = 1.0;
    e = cudaMemcpyAsync(a + root, &one, sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    for (int it = 0; it < LAP_CV_ABSORB_ITERS; ++it) {
        neighbour_sum_kernel<<<grid, kBlock, 0, st>>>(rowinfo, col, n, a, b, root);
        double *t = a; a = b; b = t;
    }
    feat_assemble<<<grid, kBlock, 0, st>>>(rowinfo, hops, n, s1, s2, ones, a, feat);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);   // the host constant above must outlive the copy
}

cudaError_t lap_launch_potential(const int2 *rowinfo, const int32_t *col, int32_t n, const double *phi, long long *h,
                                 long long *S, cudaStream_t st)
{
    const int grid = grid_for(n);
    quantize_kernel<<<grid, kBlock, 0, st>>>(phi, n, h);
    int_neighbour_sum_kernel<<<grid, kBlock, 0, st>>>(rowinfo, col, n, h, S);
    return cudaGetLastError();
}

cudaError_t lap_launch_hitting_walks(const LapDevGraph &g, int32_t root, uint64_t seed, uint32_t reps, uint64_t limit,
                                     unsigned long long *sums, unsigned int *status, int num_sms, cudaStream_t st)
{
    const uint64_t total = (uint64_t)g.n * reps;
    uint64_t grid = (total + 127) / 128;
    const uint64_t cap = (uint64_t)(num_sms > 0 ? num_sms : 1) * 16;
    if (grid > cap) grid = cap;
    hitting_walks_kernel<<<(unsigned)(grid < 1 ? 1 : grid), 128, 0, st>>>(g, root, seed, reps, limit, sums, status);
    return cudaGetLastError();
}

cudaError_t lap_launch_cv_finalize(const int2 *rowinfo, int32_t n, int32_t root, uint64_t omega,
                                   const unsigned long long *rep1, const unsigned long long *cnt2,
                                   const long long *a1, const long long *S1, double beta1,
                                   const long long *a2, const long long *p2, const long long *S2,
                                   double *ldiag, double *ecc, double *red /* kParts + 4 */, double *m2_out,
                                   cudaStream_t st)
{
    const double w = (double)omega;
    const int64_t chunk = ((int64_t)n + kParts - 1) / kParts;
    double *part = red, *s2 = red + kParts, *tr = red + kParts + 1;
    cv_y2_partial<<<kParts, kBlock, 0, st>>>(rowinfo, n, w, cnt2, chunk, part);
    total_kernel<<<1, kBlock, 0, st>>>(part, kParts, s2);
    cv_ldiag_kernel<<<grid_for(n), kBlock, 0, st>>>(rowinfo, n, root, w, (unsigned long long)omega, rep1, cnt2, a1, S1,
                                                    beta1, s2, ldiag);
    ld_partial<<<kParts, kBlock, 0, st>>>(n, ldiag, chunk, part);
    total_kernel<<<1, kBlock, 0, st>>>(part, kParts, tr);
    cv_ecc_kernel<<<grid_for(n), kBlock, 0, st>>>(n, ldiag, tr, ecc);
    if (a2) {
        m2_partial_kernel<<<kParts, kBlock, 0, st>>>(rowinfo, n, a2, p2, S2, chunk, part);
        total_kernel<<<1, kBlock, 0, st>>>(part, kParts, m2_out);
    }
    return cudaGetLastError();
}
