// MLP of the learned control variate: 8 features -> 64 -> 64 -> 2 (ReLU),
// BF16 operands on the tensor cores (mma.sync m16n8k16, FP32 accumulation),
// forward for inference, forward + MSE loss + backward for training, and
// AdamW on FP32 master weights.  (The paper has no learned component.)
//
// Parameters are one packed FP32 vector (LAP_MLP_PARAMS floats):
//   W1 [64][8] | b1 [64] | W2 [64][64] | b2 [64] | W3 [2][64] | b3 [2]
// (row = output unit).  Kernels round weights, inputs and hidden activations
// to BF16 where they enter a tensor-core product; biases, accumulators and
// gradients stay FP32.
//
// A CTA is 4 warps over blocks of 64 rows (nodes), one 16-row tile per warp.
// The forward keeps every layer in registers: the C fragment of one layer's
// m16n8 products is exactly the A fragment of the next layer's m16k16
// operand.  The backward computes dY, dH2 = dY W3 and dH1 = dH2 W2 the same
// way, stages the tiles transposed ([unit][row]) in shared memory, and forms
// the weight gradients dW = (dZ)^T A as tensor-core products over the 64 rows
// of the block (warp w owns output units 16w..16w+15), accumulating in
// registers across blocks and adding them to the global gradient once.
#include <cuda_bf16.h>

#include "lap_internal.h"

namespace {

constexpr int kIn = 8, kHid = 64, kOut = 2;
constexpr int oW1 = 0, ob1 = oW1 + kHid * kIn, oW2 = ob1 + kHid, ob2 = oW2 + kHid * kHid, oW3 = ob2 + kHid,
              ob3 = oW3 + kOut * kHid, kParams = ob3 + kOut;
static_assert(kParams == LAP_MLP_PARAMS, "packed parameter layout");

constexpr int kThreads = 128;   // 4 warps
constexpr int kRows = 64;       // rows per block
constexpr int LD1 = 24;         // padded row lengths (bf16 elements) to spread banks
constexpr int LD2 = 72;
constexpr int LD3 = 8;

// Shared memory layout (bf16 unless noted).
struct Smem {
    __nv_bfloat16 w1[kHid * LD1];     // W1 [64][24]: k 0..7 real
    __nv_bfloat16 w2[kHid * LD2];     // W2 [64][72]
    __nv_bfloat16 w2t[kHid * LD2];    // W2^T
    __nv_bfloat16 w3[8 * LD2];        // W3 [8][72]: rows 0..1 real
    __nv_bfloat16 w3t[kHid * LD3];    // W3^T [64][8]: cols 0..1 real
    float b1[kHid], b2[kHid], b3[8];
    __nv_bfloat16 xt[16 * LD2];       // X^T   [16][rows]   (features 0..7 real)
    __nv_bfloat16 h1t[kHid * LD2];    // H1^T  [64][rows]
    __nv_bfloat16 h2t[kHid * LD2];    // H2^T
    __nv_bfloat16 dh1t[kHid * LD2];   // dH1^T
    __nv_bfloat16 dh2t[kHid * LD2];   // dH2^T
    __nv_bfloat16 dyt[8 * LD2];       // dY^T  [8][rows]   (outputs 0..1 real)
    float gb1[kHid], gb2[kHid], gb3[8];
    float loss;
};

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ uint32_t ld2(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ void mma(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ void load_weights(Smem &s, const float *__restrict__ P)
{
    for (int i = threadIdx.x; i < kHid * LD1; i += kThreads) {
        const int r = i / LD1, c = i % LD1;
        s.w1[i] = __float2bfloat16_rn(c < kIn ? P[oW1 + r * kIn + c] : 0.f);
    }
    for (int i = threadIdx.x; i < kHid * LD2; i += kThreads) {
        const int r = i / LD2, c = i % LD2;
        s.w2[i] = __float2bfloat16_rn(c < kHid ? P[oW2 + r * kHid + c] : 0.f);
        s.w2t[i] = __float2bfloat16_rn(c < kHid ? P[oW2 + c * kHid + r] : 0.f);
    }
    for (int i = threadIdx.x; i < 8 * LD2; i += kThreads) {
        const int r = i / LD2, c = i % LD2;
        s.w3[i] = __float2bfloat16_rn(r < kOut && c < kHid ? P[oW3 + r * kHid + c] : 0.f);
    }
    for (int i = threadIdx.x; i < kHid * LD3; i += kThreads) {
        const int r = i / LD3, c = i % LD3;
        s.w3t[i] = __float2bfloat16_rn(c < kOut ? P[oW3 + c * kHid + r] : 0.f);
    }
    for (int i = threadIdx.x; i < kHid; i += kThreads) {
        s.b1[i] = P[ob1 + i];
        s.b2[i] = P[ob2 + i];
        s.gb1[i] = 0.f;
        s.gb2[i] = 0.f;
    }
    if (threadIdx.x < 8) {
        s.b3[threadIdx.x] = threadIdx.x < kOut ? P[ob3 + threadIdx.x] : 0.f;
        s.gb3[threadIdx.x] = 0.f;
    }
    if (threadIdx.x == 0) s.loss = 0.f;
}

template <bool TRAIN>
__global__ void __launch_bounds__(kThreads) mlp_kernel(const float *__restrict__ P, const float *__restrict__ X,
                                                       const float *__restrict__ T, int64_t n, float wk0, float wk1,
                                                       float inv_n, float *__restrict__ Y, float *__restrict__ G,
                                                       float *__restrict__ loss)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem &s = *reinterpret_cast<Smem *>(smem_raw);
    load_weights(s, P);
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
    float gw2[8][4] = {}, gw1[2][4] = {}, gw3[4] = {};   // weight-gradient accumulators (TRAIN)

    for (int64_t blk = blockIdx.x; blk * kRows < n; blk += gridDim.x) {
        const int64_t r0 = blk * kRows + warp * 16;
        const int64_t ra = r0 + gid, rb = r0 + gid + 8;
        const bool va = ra < n, vb = rb < n;

        // ---- layer 1: X [16 x 16 (8 real)] x W1^T
        uint32_t ax[4];
        {
            const float2 xa = va ? *reinterpret_cast<const float2 *>(X + ra * kIn + 2 * tig) : make_float2(0.f, 0.f);
            const float2 xb = vb ? *reinterpret_cast<const float2 *>(X + rb * kIn + 2 * tig) : make_float2(0.f, 0.f);
            ax[0] = pack2(xa.x, xa.y);
            ax[1] = pack2(xb.x, xb.y);
            ax[2] = 0u;
            ax[3] = 0u;
        }
        float h1[8][4];
        uint32_t m1 = 0;   // ReLU masks, bit 4j+q for h1[j][q]
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            const __nv_bfloat16 *wp = s.w1 + (j * 8 + gid) * LD1 + 2 * tig;
            mma(c, ax, ld2(wp), ld2(wp + 8));
            const float bb0 = s.b1[j * 8 + 2 * tig], bb1 = s.b1[j * 8 + 2 * tig + 1];
            c[0] += bb0; c[1] += bb1; c[2] += bb0; c[3] += bb1;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (c[q] > 0.f) m1 |= 1u << (4 * j + q);
                h1[j][q] = fmaxf(c[q], 0.f);
            }
        }
        // ---- layer 2: H1 [16 x 64] x W2^T
        uint32_t ah[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ah[k][0] = pack2(h1[2 * k][0], h1[2 * k][1]);
            ah[k][1] = pack2(h1[2 * k][2], h1[2 * k][3]);
            ah[k][2] = pack2(h1[2 * k + 1][0], h1[2 * k + 1][1]);
            ah[k][3] = pack2(h1[2 * k + 1][2], h1[2 * k + 1][3]);
        }
        float h2[8][4];
        uint32_t m2 = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const __nv_bfloat16 *wp = s.w2 + (j * 8 + gid) * LD2 + k * 16 + 2 * tig;
                mma(c, ah[k], ld2(wp), ld2(wp + 8));
            }
            const float bb0 = s.b2[j * 8 + 2 * tig], bb1 = s.b2[j * 8 + 2 * tig + 1];
            c[0] += bb0; c[1] += bb1; c[2] += bb0; c[3] += bb1;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (c[q] > 0.f) m2 |= 1u << (4 * j + q);
                h2[j][q] = fmaxf(c[q], 0.f);
            }
        }
        // ---- layer 3: H2 [16 x 64] x W3^T (2 real outputs of 8)
        uint32_t ag[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ag[k][0] = pack2(h2[2 * k][0], h2[2 * k][1]);
            ag[k][1] = pack2(h2[2 * k][2], h2[2 * k][3]);
            ag[k][2] = pack2(h2[2 * k + 1][0], h2[2 * k + 1][1]);
            ag[k][3] = pack2(h2[2 * k + 1][2], h2[2 * k + 1][3]);
        }
        float y[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __nv_bfloat16 *wp = s.w3 + gid * LD2 + k * 16 + 2 * tig;
            mma(y, ag[k], ld2(wp), ld2(wp + 8));
        }
        if (tig == 0) {
            y[0] += s.b3[0]; y[1] += s.b3[1]; y[2] += s.b3[0]; y[3] += s.b3[1];
        }
        if (!TRAIN) {
            if (tig == 0) {
                if (va) *reinterpret_cast<float2 *>(Y + ra * kOut) = make_float2(y[0], y[1]);
                if (vb) *reinterpret_cast<float2 *>(Y + rb * kOut) = make_float2(y[2], y[3]);
            }
            continue;
        }

        // ---- loss and dY = 2 w_k (y - t) / N (rows beyond n contribute nothing)
        float dy[4] = {0.f, 0.f, 0.f, 0.f};
        if (tig == 0) {
            float lsum = 0.f;
            if (va) {
                const float2 t = *reinterpret_cast<const float2 *>(T + ra * kOut);
                const float e0 = y[0] - t.x, e1 = y[1] - t.y;
                dy[0] = 2.f * wk0 * e0 * inv_n;
                dy[1] = 2.f * wk1 * e1 * inv_n;
                lsum += wk0 * e0 * e0 + wk1 * e1 * e1;
            }
            if (vb) {
                const float2 t = *reinterpret_cast<const float2 *>(T + rb * kOut);
                const float e0 = y[2] - t.x, e1 = y[3] - t.y;
                dy[2] = 2.f * wk0 * e0 * inv_n;
                dy[3] = 2.f * wk1 * e1 * inv_n;
                lsum += wk0 * e0 * e0 + wk1 * e1 * e1;
            }
            atomicAdd(&s.loss, lsum * inv_n);
            atomicAdd(&s.gb3[0], dy[0] + dy[2]);
            atomicAdd(&s.gb3[1], dy[1] + dy[3]);
        }
        // Stage X^T, H1^T, H2^T, dY^T (BF16, as used by the products).
        const int ca = warp * 16 + gid, cb = ca + 8;     // row index inside the block
        {
            const float2 xa = va ? *reinterpret_cast<const float2 *>(X + ra * kIn + 2 * tig) : make_float2(0.f, 0.f);
            const float2 xb = vb ? *reinterpret_cast<const float2 *>(X + rb * kIn + 2 * tig) : make_float2(0.f, 0.f);
            s.xt[(2 * tig) * LD2 + ca] = __float2bfloat16_rn(xa.x);
            s.xt[(2 * tig + 1) * LD2 + ca] = __float2bfloat16_rn(xa.y);
            s.xt[(2 * tig) * LD2 + cb] = __float2bfloat16_rn(xb.x);
            s.xt[(2 * tig + 1) * LD2 + cb] = __float2bfloat16_rn(xb.y);
            s.xt[(8 + 2 * tig) * LD2 + ca] = __float2bfloat16_rn(0.f);
            s.xt[(9 + 2 * tig) * LD2 + ca] = __float2bfloat16_rn(0.f);
            s.xt[(8 + 2 * tig) * LD2 + cb] = __float2bfloat16_rn(0.f);
            s.xt[(9 + 2 * tig) * LD2 + cb] = __float2bfloat16_rn(0.f);
            s.dyt[(2 * tig) * LD2 + ca] = __float2bfloat16_rn(dy[0]);
            s.dyt[(2 * tig + 1) * LD2 + ca] = __float2bfloat16_rn(dy[1]);
            s.dyt[(2 * tig) * LD2 + cb] = __float2bfloat16_rn(dy[2]);
            s.dyt[(2 * tig + 1) * LD2 + cb] = __float2bfloat16_rn(dy[3]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int u0 = j * 8 + 2 * tig, u1 = u0 + 1;
            s.h1t[u0 * LD2 + ca] = __float2bfloat16_rn(h1[j][0]);
            s.h1t[u1 * LD2 + ca] = __float2bfloat16_rn(h1[j][1]);
            s.h1t[u0 * LD2 + cb] = __float2bfloat16_rn(h1[j][2]);
            s.h1t[u1 * LD2 + cb] = __float2bfloat16_rn(h1[j][3]);
            s.h2t[u0 * LD2 + ca] = __float2bfloat16_rn(h2[j][0]);
            s.h2t[u1 * LD2 + ca] = __float2bfloat16_rn(h2[j][1]);
            s.h2t[u0 * LD2 + cb] = __float2bfloat16_rn(h2[j][2]);
            s.h2t[u1 * LD2 + cb] = __float2bfloat16_rn(h2[j][3]);
        }
        // ---- dH2 = (dY W3) * relu'(Z2): dY as the A operand (cols 0..7 of 16).
        uint32_t ad[4] = {pack2(dy[0], dy[1]), pack2(dy[2], dy[3]), 0u, 0u};
        float dh2[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
            mma(c, ad, ld2(s.w3t + (j * 8 + gid) * LD3 + 2 * tig), 0u);
            float cs0 = 0.f, cs1 = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                dh2[j][q] = (m2 >> (4 * j + q)) & 1u ? c[q] : 0.f;
            }
            cs0 = dh2[j][0] + dh2[j][2];
            cs1 = dh2[j][1] + dh2[j][3];
            atomicAdd(&s.gb2[j * 8 + 2 * tig], cs0);
            atomicAdd(&s.gb2[j * 8 + 2 * tig + 1], cs1);
            const int u0 = j * 8 + 2 * tig, u1 = u0 + 1;
            s.dh2t[u0 * LD2 + ca] = __float2bfloat16_rn(dh2[j][0]);
            s.dh2t[u1 * LD2 + ca] = __float2bfloat16_rn(dh2[j][1]);
            s.dh2t[u0 * LD2 + cb] = __float2bfloat16_rn(dh2[j][2]);
            s.dh2t[u1 * LD2 + cb] = __float2bfloat16_rn(dh2[j][3]);
        }
        // ---- dH1 = (dH2 W2) * relu'(Z1)
        uint32_t ae[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ae[k][0] = pack2(dh2[2 * k][0], dh2[2 * k][1]);
            ae[k][1] = pack2(dh2[2 * k][2], dh2[2 * k][3]);
            ae[k][2] = pack2(dh2[2 * k + 1][0], dh2[2 * k + 1][1]);
            ae[k][3] = pack2(dh2[2 * k + 1][2], dh2[2 * k + 1][3]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const __nv_bfloat16 *wp = s.w2t + (j * 8 + gid) * LD2 + k * 16 + 2 * tig;
                mma(c, ae[k], ld2(wp), ld2(wp + 8));
            }
            float d[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) d[q] = (m1 >> (4 * j + q)) & 1u ? c[q] : 0.f;
            atomicAdd(&s.gb1[j * 8 + 2 * tig], d[0] + d[2]);
            atomicAdd(&s.gb1[j * 8 + 2 * tig + 1], d[1] + d[3]);
            const int u0 = j * 8 + 2 * tig, u1 = u0 + 1;
            s.dh1t[u0 * LD2 + ca] = __float2bfloat16_rn(d[0]);
            s.dh1t[u1 * LD2 + ca] = __float2bfloat16_rn(d[1]);
            s.dh1t[u0 * LD2 + cb] = __float2bfloat16_rn(d[2]);
            s.dh1t[u1 * LD2 + cb] = __float2bfloat16_rn(d[3]);
        }
        __syncthreads();
        // ---- weight gradients over the 64 rows of the block; warp w owns
        // output units 16w..16w+15 of W2 and W1 and hidden units of W3^T.
        const int mrow = warp * 16 + gid;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t a2[4], a1[4], a3[4];
            const __nv_bfloat16 *p2 = s.dh2t + mrow * LD2 + k * 16 + 2 * tig;
            a2[0] = ld2(p2); a2[1] = ld2(p2 + 8 * LD2); a2[2] = ld2(p2 + 8); a2[3] = ld2(p2 + 8 * LD2 + 8);
            const __nv_bfloat16 *p1 = s.dh1t + mrow * LD2 + k * 16 + 2 * tig;
            a1[0] = ld2(p1); a1[1] = ld2(p1 + 8 * LD2); a1[2] = ld2(p1 + 8); a1[3] = ld2(p1 + 8 * LD2 + 8);
            const __nv_bfloat16 *p3 = s.h2t + mrow * LD2 + k * 16 + 2 * tig;
            a3[0] = ld2(p3); a3[1] = ld2(p3 + 8 * LD2); a3[2] = ld2(p3 + 8); a3[3] = ld2(p3 + 8 * LD2 + 8);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const __nv_bfloat16 *bp = s.h1t + (j * 8 + gid) * LD2 + k * 16 + 2 * tig;
                mma(gw2[j], a2, ld2(bp), ld2(bp + 8));
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const __nv_bfloat16 *bp = s.xt + (j * 8 + gid) * LD2 + k * 16 + 2 * tig;
                mma(gw1[j], a1, ld2(bp), ld2(bp + 8));
            }
            const __nv_bfloat16 *bp = s.dyt + gid * LD2 + k * 16 + 2 * tig;
            mma(gw3, a3, ld2(bp), ld2(bp + 8));
        }
        __syncthreads();
    }
    if (!TRAIN) return;

    // ---- add this CTA's gradients to the global FP32 gradient
    const int mrow = warp * 16 + gid;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c0 = j * 8 + 2 * tig;
        atomicAdd(&G[oW2 + mrow * kHid + c0], gw2[j][0]);
        atomicAdd(&G[oW2 + mrow * kHid + c0 + 1], gw2[j][1]);
        atomicAdd(&G[oW2 + (mrow + 8) * kHid + c0], gw2[j][2]);
        atomicAdd(&G[oW2 + (mrow + 8) * kHid + c0 + 1], gw2[j][3]);
    }
    {
        const int c0 = 2 * tig;   // input features 0..7 are n-tile 0
        atomicAdd(&G[oW1 + mrow * kIn + c0], gw1[0][0]);
        atomicAdd(&G[oW1 + mrow * kIn + c0 + 1], gw1[0][1]);
        atomicAdd(&G[oW1 + (mrow + 8) * kIn + c0], gw1[0][2]);
        atomicAdd(&G[oW1 + (mrow + 8) * kIn + c0 + 1], gw1[0][3]);
    }
    if (tig == 0) {   // W3^T columns 0..1 = outputs
        atomicAdd(&G[oW3 + 0 * kHid + mrow], gw3[0]);
        atomicAdd(&G[oW3 + 1 * kHid + mrow], gw3[1]);
        atomicAdd(&G[oW3 + 0 * kHid + mrow + 8], gw3[2]);
        atomicAdd(&G[oW3 + 1 * kHid + mrow + 8], gw3[3]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHid; i += kThreads) {
        atomicAdd(&G[ob1 + i], s.gb1[i]);
        atomicAdd(&G[ob2 + i], s.gb2[i]);
    }
    if (threadIdx.x < kOut) atomicAdd(&G[ob3 + threadIdx.x], s.gb3[threadIdx.x]);
    if (threadIdx.x == 0) atomicAdd(loss, s.loss);
}

// AdamW with decoupled weight decay (Loshchilov & Hutter) on FP32 masters.
__global__ void adamw_kernel(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                             const float *__restrict__ g, int64_t count, float lr, float b1, float b2, float eps,
                             float wd, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float mh = mi / c1, vh = vi / c2;
        w[i] = w[i] - lr * (mh / (sqrtf(vh) + eps) + wd * w[i]);
    }
}

int grid_for(int64_t n, int num_sms)
{
    int64_t blocks = (n + kRows - 1) / kRows;
    const int64_t cap = (int64_t)(num_sms > 0 ? num_sms : 1) * 4;
    if (blocks > cap) blocks = cap;
    return (int)(blocks < 1 ? 1 : blocks);
}

int current_sms()
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

cudaError_t lap_launch_mlp_mma_sync(const float *P, const float *X, const float *T, int64_t n, float wk0,
                                     float wk1, float *Y, float *G, float *loss, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const size_t smem = sizeof(Smem);
    const int grid = grid_for(n, current_sms());
    if (T) {
        cudaError_t e = cudaFuncSetAttribute(mlp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        mlp_kernel<true><<<grid, kThreads, smem, st>>>(P, X, T, n, wk0, wk1, 1.f / (float)n, Y, G, loss);
    } else {
        cudaError_t e = cudaFuncSetAttribute(mlp_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        mlp_kernel<false><<<grid, kThreads, smem, st>>>(P, X, nullptr, n, 0.f, 0.f, 0.f, Y, nullptr, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t lap_launch_adamw(float *w, float *m, float *v, const float *g, int64_t count, int32_t step, float lr,
                             float b1, float b2, float eps, float wd, cudaStream_t st)
{
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    const int grid = (int)((count + 255) / 256 > 1024 ? 1024 : (count + 255) / 256);
    adamw_kernel<<<grid < 1 ? 1 : grid, 256, 0, st>>>(w, m, v, g, count, lr, b1, b2, eps, wd, c1, c2);
    return cudaGetLastError();
}
