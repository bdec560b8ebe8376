// Control-variate support kernels (the paper has no control variate; see
// include/lap.h, lap_features .. lap_cv_estimates):
//   * 8 local node features for the MLP,
//   * integer potentials h = round(2^16 phi) and neighbour sums S[u],
//   * hitting-time targets: v-absorbed walks from every node (Section 3.2,
//     v-absorbed walk lemma: E[length from u] = h(u, v) = (L_v^{-1} d)_u),
//   * the CV finalize: Z1[u] = d_u A1[u] - cnt1[u] S1[u] and
//     M2 = sum_u (d_u A2[u] - P2[u] S2[u]) / d_u, then
//     y1_cv(u) = (cnt1[u] - beta1 Z1[u] / d_u) / (omega d_u) and
//     kappa_cv = (sum Y1 - sum Y2 + beta2 M2) / omega,
//   * the network's training targets and the potentials from its outputs,
//   * the coefficients beta1, beta2 from pilot batches (least squares).
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

// Training targets of one graph from its counts: t0 = cnt1 / omega (mean
// Wilson visits, d_u (L_v^{-1})_uu), t1 = (hitting-walk sum / reps) / mean_y2
// (h(u, v) / E[Y2]); both zero at the root.
__global__ void cv_targets_kernel(int32_t n, int32_t root, unsigned long long omega_u, double omega,
                                  const unsigned long long *__restrict__ rep1,
                                  const unsigned long long *__restrict__ hit, double reps, double mean_y2,
                                  float2 *__restrict__ t)
{
    NODE_LOOP(u, n)
    {
        if (u == root) { t[u] = make_float2(0.f, 0.f); continue; }
        const double t0 = __ddiv_rn((double)(omega_u + rep1[u]), omega);
        const double t1 = __ddiv_rn(__ddiv_rn((double)hit[u], reps), mean_y2);
        t[u] = make_float2((float)t0, (float)t1);
    }
}

// Potentials from the network's outputs y[u] = (pred visits, pred hitting
// time / E[Y2]): phi1 = y0 / d_u ~ (L_v^{-1})_uu, phi2 = y1 * scale2 ~ h(u, v),
// phi2(root) = 0.
__global__ void cv_potentials_kernel(const int2 *__restrict__ rowinfo, int32_t n, int32_t root,
                                     const float2 *__restrict__ y, double scale2, double *__restrict__ phi1,
                                     double *__restrict__ phi2)
{
    NODE_LOOP(u, n)
    {
        const float2 o = y[u];
        if (phi1) phi1[u] = __ddiv_rn((double)o.x, (double)rowinfo[u].y);
        if (phi2) phi2[u] = (u == root) ? 0.0 : __dmul_rn((double)o.y, scale2);
    }
}

// One pilot batch of the beta1 fit: the batch's visits V(u) (difference of the
// cumulative cnt1 = omega + rep1) and its martingale sum Z1(u) / d_u, with
// Z1 = d_u dA1(u) - dV(u) S1(u) in exact int64 arithmetic; the cumulative
// values are kept for the next batch.
__global__ void beta1_batch_kernel(const int2 *__restrict__ rowinfo, int32_t n, int32_t root,
                                   unsigned long long omega_u, const unsigned long long *__restrict__ rep1,
                                   const long long *__restrict__ a1, const long long *__restrict__ S1,
                                   long long *__restrict__ prev_c1, long long *__restrict__ prev_a1,
                                   double *__restrict__ vb, double *__restrict__ zb)
{
    NODE_LOOP(u, n)
    {
        if (u == root) { vb[u] = 0.0; zb[u] = 0.0; continue; }
        const long long c1 = (long long)(omega_u + rep1[u]), a = a1[u];
        const long long dv = c1 - prev_c1[u], da = a - prev_a1[u];
        prev_c1[u] = c1;
        prev_a1[u] = a;
        const long long d = rowinfo[u].y;
        vb[u] = (double)dv;
        zb[u] = __ddiv_rn((double)(d * da - dv * S1[u]), (double)d);
    }
}

// beta1 = sum_u sum_b (V_bu - mean_b V_bu)(Z_bu - mean_b Z_bu) /
//         sum_u sum_b (Z_bu - mean_b Z_bu)^2   (pooled over nodes): per
// node the two centred sums over the B batches, partial sums per chunk.
__global__ void beta1_partial(int32_t n, int32_t batches, const double *__restrict__ vb, const double *__restrict__ zb,
                              int64_t chunk, double *__restrict__ part_num, double *__restrict__ part_den)
{
    const int64_t a = (int64_t)blockIdx.x * chunk;
    const int64_t b = a + chunk < n ? a + chunk : n;
    double num = 0.0, den = 0.0;
    const double inv_b = __ddiv_rn(1.0, (double)batches);
    for (int64_t u = a + threadIdx.x; u < b; u += kBlock) {
        double mv = 0.0, mz = 0.0;
        for (int32_t k = 0; k < batches; ++k) {
            mv = __dadd_rn(mv, vb[(int64_t)k * n + u]);
            mz = __dadd_rn(mz, zb[(int64_t)k * n + u]);
        }
        mv = __dmul_rn(mv, inv_b);
        mz = __dmul_rn(mz, inv_b);
        for (int32_t k = 0; k < batches; ++k) {
            const double cv = __dsub_rn(vb[(int64_t)k * n + u], mv), cz = __dsub_rn(zb[(int64_t)k * n + u], mz);
            num = __dadd_rn(num, __dmul_rn(cv, cz));
            den = __dadd_rn(den, __dmul_rn(cz, cz));
        }
    }
    num = block_sum(num);
    den = block_sum(den);
    if (threadIdx.x == 0) {
        part_num[blockIdx.x] = num;
        part_den[blockIdx.x] = den;
    }
}

// beta2 from the per-sample traces y_k = Y1_k - Y2_k and m_k = M2_k:
// beta2 = -cov(y, m) / var(m).  Pass 1: partial sums of y and m; pass 2:
// partial centred sums of (y - ybar)(m - mbar) and (m - mbar)^2.
__device__ __forceinline__ double trace_y(const unsigned long long *y1, const unsigned long long *y2, int64_t k)
{
    return (double)(long long)(y1[k] - y2[k]);
}

__global__ void trace_sum_partial(const unsigned long long *__restrict__ y1, const unsigned long long *__restrict__ y2,
                                  const double *__restrict__ m2, int64_t count, int64_t chunk,
                                  double *__restrict__ part_y, double *__restrict__ part_m)
{
    const int64_t a = (int64_t)blockIdx.x * chunk;
    const int64_t b = a + chunk < count ? a + chunk : count;
    double sy = 0.0, sm = 0.0;
    for (int64_t k = a + threadIdx.x; k < b; k += kBlock) {
        sy = __dadd_rn(sy, trace_y(y1, y2, k));
        sm = __dadd_rn(sm, m2[k]);
    }
    sy = block_sum(sy);
    sm = block_sum(sm);
    if (threadIdx.x == 0) {
        part_y[blockIdx.x] = sy;
        part_m[blockIdx.x] = sm;
    }
}

__global__ void trace_cov_partial(const unsigned long long *__restrict__ y1, const unsigned long long *__restrict__ y2,
                                  const double *__restrict__ m2, int64_t count, int64_t chunk, const double *sums,
                                  double *__restrict__ part_c, double *__restrict__ part_v)
{
    const double my = __ddiv_rn(sums[0], (double)count), mm = __ddiv_rn(sums[1], (double)count);
    const int64_t a = (int64_t)blockIdx.x * chunk;
    const int64_t b = a + chunk < count ? a + chunk : count;
    double c = 0.0, v = 0.0;
    for (int64_t k = a + threadIdx.x; k < b; k += kBlock) {
        const double dy = __dsub_rn(trace_y(y1, y2, k), my), dm = __dsub_rn(m2[k], mm);
        c = __dadd_rn(c, __dmul_rn(dy, dm));
        v = __dadd_rn(v, __dmul_rn(dm, dm));
    }
    c = block_sum(c);
    v = block_sum(v);
    if (threadIdx.x == 0) {
        part_c[blockIdx.x] = c;
        part_v[blockIdx.x] = v;
    }
}

}  // namespace

cudaError_t lap_launch_cv_targets(int32_t n, int32_t root, uint64_t omega, const unsigned long long *rep1,
                                  const unsigned long long *hit, uint32_t reps, double mean_y2, float *targets,
                                  cudaStream_t st)
{
    cv_targets_kernel<<<grid_for(n), kBlock, 0, st>>>(n, root, (unsigned long long)omega, (double)omega, rep1, hit,
                                                      (double)reps, mean_y2, reinterpret_cast<float2 *>(targets));
    return cudaGetLastError();
}

cudaError_t lap_launch_cv_potentials(const int2 *rowinfo, int32_t n, int32_t root, const float *y, double scale2,
                                     double *phi1, double *phi2, cudaStream_t st)
{
    cv_potentials_kernel<<<grid_for(n), kBlock, 0, st>>>(rowinfo, n, root, reinterpret_cast<const float2 *>(y), scale2,
                                                         phi1, phi2);
    return cudaGetLastError();
}

cudaError_t lap_launch_beta1_batch(const int2 *rowinfo, int32_t n, int32_t root, uint64_t omega,
                                   const unsigned long long *rep1, const long long *a1, const long long *S1,
                                   long long *prev_c1, long long *prev_a1, double *vb, double *zb, cudaStream_t st)
{
    beta1_batch_kernel<<<grid_for(n), kBlock, 0, st>>>(rowinfo, n, root, (unsigned long long)omega, rep1, a1, S1,
                                                       prev_c1, prev_a1, vb, zb);
    return cudaGetLastError();
}

// red: at least 2 * kParts + 4 doubles; out[0] = numerator, out[1] = denominator.
cudaError_t lap_launch_beta1_reduce(int32_t n, int32_t batches, const double *vb, const double *zb, double *red,
                                    double *out, cudaStream_t st)
{
    const int64_t chunk = ((int64_t)n + kParts - 1) / kParts;
    beta1_partial<<<kParts, kBlock, 0, st>>>(n, batches, vb, zb, chunk, red, red + kParts);
    total_kernel<<<1, kBlock, 0, st>>>(red, kParts, out);
    total_kernel<<<1, kBlock, 0, st>>>(red + kParts, kParts, out + 1);
    return cudaGetLastError();
}

// red: at least 2 * kParts + 4 doubles; out[0] = cov numerator, out[1] = var
// numerator (both before dividing by count - 1).
cudaError_t lap_launch_beta2_reduce(const unsigned long long *y1, const unsigned long long *y2, const double *m2,
                                    int64_t count, double *red, double *out, cudaStream_t st)
{
    const int64_t chunk = (count + kParts - 1) / kParts;
    double *sums = red + 2 * kParts;
    trace_sum_partial<<<kParts, kBlock, 0, st>>>(y1, y2, m2, count, chunk, red, red + kParts);
    total_kernel<<<1, kBlock, 0, st>>>(red, kParts, sums);
    total_kernel<<<1, kBlock, 0, st>>>(red + kParts, kParts, sums + 1);
    trace_cov_partial<<<kParts, kBlock, 0, st>>>(y1, y2, m2, count, chunk, sums, red, red + kParts);
    total_kernel<<<1, kBlock, 0, st>>>(red, kParts, out);
    total_kernel<<<1, kBlock, 0, st>>>(red + kParts, kParts, out + 1);
    return cudaGetLastError();
}

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
