// Compact LEWalk sampler: same computation and same counts as lewalk_kernel
// (sampler.cu: Wilson LE_v run, uniform-start and pi-start v-absorbed walks
// per sample; Alg. 2 and Alg. 4), with one byte of state per node per sample
// in flight instead of eight, so about eight times more samples (independent
// gather chains) fit in HBM.
//
// Per node and sample one byte:   bit 7 epoch | bit 6 InTree | bit 5 OnPath | bits 0..4 draws k
// The Next[] array of Alg. 2 is replaced by a per-lane stack holding the
// current loop-erased path (entries: node | k << 27).  A walk step at head h
// draws stack entry k of h (Philox counter (h, k, i, 0)), pushes h and moves
// to w = RandomNeighbor(h):
//   w InTree  -> the path joins the tree: every stacked node is marked InTree
//                (Alg. 2's retrace; the path on the stack is exactly the
//                loop-erased path the retrace would follow along Next[]);
//   w OnPath  -> the walk closed a loop at w: the nodes above w are erased
//                (OnPath cleared, their draw counts kept) and w draws again;
//   otherwise -> w becomes the head.
// Visits, Y1 and the tree are those of the sequential run, because every
// draw is still the next entry of the node's stack.
//
// Every node's byte keeps its draw count k for the whole sample (also once
// InTree), and the repeat-visit counter has received exactly k - 1 for every
// node touched so far.  A sample that cannot be represented (a node drawn
// more than 31 times, or a loop-erased path longer than the stack) is
// therefore withdrawn exactly: the lane subtracts k - 1 for every node of
// the sample, re-stamps its state bytes with the current epoch (so the next
// sample sees them all as stale), appends the sample id to an overflow list
// and goes on with the next sample.  The host re-runs the listed ids with
// the 8-byte kernel.  Nothing else of a sample is counted before its Wilson
// run completes.
#include "lap_internal.h"
#include "philox.cuh"

namespace {

constexpr uint32_t kBEpoch = 0x80u, kBTree = 0x40u, kBPath = 0x20u, kBK = 0x1Fu;
constexpr uint32_t kKMax = 31u;
constexpr int kEntryShift = 27;
constexpr uint32_t kNodeMask = (1u << kEntryShift) - 1u;

// Phases of a lane.  Each loop iteration issues at most one round of
// dependent loads per lane; the *_IMMEDIATE phases are transitions that need
// no load and run in the same iteration.
enum Phase : uint32_t {
    P_CLAIM = 0,
    P_WALK,                // pa = state byte of the head h, pb = row record of h
    P_SCAN,                // pq = 16 state bytes at `chunk`
    P_USTART_IMMEDIATE,
    P_UWALK,               // pb = row record of the walk's node (uniform start)
    P_PISTART_IMMEDIATE,
    P_PIWALK,              // pb = row record of the walk's node (pi start)
    P_FINISH_IMMEDIATE
};

// L2 eviction policies (sm_80+ createpolicy) and loads/stores that use them.
__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// State bytes: default L2 priority (a sector read at one step is written at
// the next step and again at the retrace, so it should stay in L2 meanwhile;
// evicting it early turns those writes into partial-sector fills), no L1
// allocation (no reuse within a lane at L1 time scales).
__device__ __forceinline__ uint32_t ld_state(const uint8_t *a)
{
    uint16_t v;
    asm volatile("ld.global.L1::no_allocate.u8 %0, [%1];" : "=h"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_state(uint8_t *a, uint32_t v)
{
    asm volatile("st.global.L1::no_allocate.u8 [%0], %1;" ::"l"(a), "h"((uint16_t)v) : "memory");
}
// Path-stack entries: kept in L2 with the graph (they are re-read at the retrace).
__device__ __forceinline__ void st_stack(uint32_t *a, uint32_t v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ int32_t ld_col(const int32_t *a, uint64_t pol)
{
    int32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ uint64_t ld_row(const int2 *rowinfo, int32_t u, uint64_t pol)
{
    uint64_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(rowinfo + u), "l"(pol));
    return v;
}

__device__ __forceinline__ bool b_current(uint32_t b, uint32_t ep) { return (b & kBEpoch) == ep; }
__device__ __forceinline__ bool b_tree(uint32_t b, uint32_t ep) { return b_current(b, ep) && (b & kBTree); }
__device__ __forceinline__ bool b_path(uint32_t b, uint32_t ep) { return b_current(b, ep) && (b & kBPath); }
__device__ __forceinline__ uint32_t b_k(uint32_t b, uint32_t ep) { return b_current(b, ep) ? (b & kBK) : 0u; }
__device__ __forceinline__ int32_t row_off(uint64_t r) { return (int32_t)(uint32_t)r; }
__device__ __forceinline__ uint32_t row_deg(uint64_t r) { return (uint32_t)(r >> 32); }

// Bit b of the result is set when byte b of the 16 bytes is not InTree
// (InTree bytes have top bits == epoch | InTree).  Per 4-byte word: SIMD byte
// compare, then bit 7 of each byte gathered into 4 bits by one multiply.
__device__ __forceinline__ uint32_t gather4(uint32_t eq) { return ((((eq >> 7) & 0x01010101u) * 0x01020408u) >> 24) & 0xFu; }
__device__ __forceinline__ uint32_t not_tree_mask(ulonglong2 q, uint32_t ep)
{
    const uint32_t want = (ep | kBTree) * 0x01010101u;
    const uint32_t w0 = (uint32_t)q.x, w1 = (uint32_t)(q.x >> 32), w2 = (uint32_t)q.y, w3 = (uint32_t)(q.y >> 32);
    const uint32_t t = gather4(__vcmpeq4(w0 & 0xC0C0C0C0u, want)) | (gather4(__vcmpeq4(w1 & 0xC0C0C0C0u, want)) << 4) |
                       (gather4(__vcmpeq4(w2 & 0xC0C0C0C0u, want)) << 8) | (gather4(__vcmpeq4(w3 & 0xC0C0C0C0u, want)) << 12);
    return ~t & 0xFFFFu;
}

// The lane keeps the 16 state bytes at `chunk` in registers (pq) as an exact
// copy: it is the only writer of its state, so every byte it writes inside
// the chunk is also written into pq.  Starts found in pq need no re-read.
__device__ __forceinline__ void pq_set(ulonglong2 &pq, int32_t chunk, uint32_t u, uint32_t b)
{
    const uint32_t off = u - (uint32_t)chunk;
    if (off < 16u) {
        const uint32_t sh = 8u * (off & 7u);
        const unsigned long long m = ~(0xFFull << sh), v = (unsigned long long)(b & 0xFFu) << sh;
        if (off < 8u) pq.x = (pq.x & m) | v;
        else pq.y = (pq.y & m) | v;
    }
}

// Marks every node on the stack InTree, keeping its draw count.  The order
// does not matter, so entries are read 16 at a time with independent vector
// loads (the stack is 16-byte aligned) instead of one dependent pop each.
__device__ __forceinline__ void commit_one(uint8_t *st, uint32_t e, uint32_t ep, ulonglong2 &pq, int32_t chunk)
{
    const uint32_t b = ep | kBTree | (e >> kEntryShift);
    st[e & kNodeMask] = (uint8_t)b;
    pq_set(pq, chunk, e & kNodeMask, b);
}
__device__ __forceinline__ void commit_path(uint8_t *st, const uint32_t *stk, uint32_t sp, uint32_t ep,
                                            ulonglong2 &pq, int32_t chunk)
{
    uint32_t j = 0;
    for (; j + 16u <= sp; j += 16u) {
        uint4 e[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) e[q] = *reinterpret_cast<const uint4 *>(stk + j + 4u * q);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            commit_one(st, e[q].x, ep, pq, chunk);
            commit_one(st, e[q].y, ep, pq, chunk);
            commit_one(st, e[q].z, ep, pq, chunk);
            commit_one(st, e[q].w, ep, pq, chunk);
        }
    }
    for (; j < sp; ++j) commit_one(st, stk[j], ep, pq, chunk);
}

// Loop closed at head h (h is on the stack): erases the entries above h
// (OnPath cleared, draw counts kept) and removes h's own entry; returns the
// new depth.  Reads the stack top down, one aligned group of 4 per load.
__device__ __forceinline__ uint32_t erase_loop(uint8_t *st, const uint32_t *stk, uint32_t sp, uint32_t ep, uint32_t h,
                                               ulonglong2 &pq, int32_t chunk)
{
    for (;;) {
        const uint32_t top = sp - 1u;
        const uint32_t g0 = top & ~3u;
        const uint4 e4 = *reinterpret_cast<const uint4 *>(stk + g0);
        const uint32_t e[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
        for (int q = 3; q >= 0; --q) {
            if ((uint32_t)q > top - g0) continue;
            const uint32_t node = e[q] & kNodeMask;
            if (node == h) return g0 + (uint32_t)q;
            st[node] = (uint8_t)(ep | (e[q] >> kEntryShift));
            pq_set(pq, chunk, node, ep | (e[q] >> kEntryShift));
        }
        sp = g0;
    }
}

// Withdraws a partly run sample: subtracts the k - 1 repeat visits every
// node of the sample has contributed (and, with the control variate, the
// potentials h1[w] of its k draws, recomputed from their Philox keys) and
// marks all bytes "current epoch, untouched", so that the next sample (next
// epoch) reads them as stale.
__device__ void withdraw_sample(uint8_t *st, int32_t n, uint32_t ep, unsigned long long *rep1, const int2 *rowinfo,
                                const int32_t *col, const long long *h1, unsigned long long *a1, uint32_t i,
                                uint32_t key0, uint32_t key1)
{
    for (int32_t base = 0; base < n; base += 16) {
        ulonglong2 q = *reinterpret_cast<ulonglong2 *>(st + base);
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            const uint32_t byte = (uint32_t)(((b < 8 ? q.x : q.y) >> (8 * (b & 7))) & 0xFFu);
            const uint32_t k = b_k(byte, ep);
            if (base + b >= n) continue;
            if (k >= 2u) atomicAdd(&rep1[base + b], (unsigned long long)(-(long long)(k - 1u)));
            if (h1 && k) {
                const int2 r = rowinfo[base + b];
                long long sub = 0;
                for (uint32_t j = 0; j < k; ++j) {
                    const uint64_t x = lap::philox_r64((uint32_t)(base + b), j, i, 0u, key0, key1);
                    sub += h1[col[r.x + (int64_t)lap::below(x, (uint64_t)r.y)]];
                }
                atomicAdd(&a1[base + b], (unsigned long long)(-sub));
            }
        }
        const unsigned long long fill = 0x0101010101010101ull * (unsigned long long)ep;
        *reinterpret_cast<ulonglong2 *>(st + base) = make_ulonglong2(fill, fill);
    }
}

template <bool CV>
__global__ void __launch_bounds__(256) lewalk_compact_kernel(LapSampleLaunch p)
{
    const uint64_t slot = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (slot >= p.slots) return;
    const int32_t n = p.g.n;
    const int32_t v = p.root;
    const int2 *__restrict__ rowinfo = p.g.rowinfo;
    const int32_t *__restrict__ col = p.g.col;
    uint8_t *__restrict__ st = reinterpret_cast<uint8_t *>(p.ws) + slot * p.slot_bytes;
    uint32_t *__restrict__ stk = reinterpret_cast<uint32_t *>(st + p.n_pad);
    const uint32_t cap = p.stack_cap;
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    const uint64_t limit = p.step_limit;
    // The graph (row records, columns) and the path stacks should stay in L2.
    const uint64_t keep = policy_evict_last();

    uint32_t ep = p.slot_epoch[slot] ? kBEpoch : 0u;
    uint32_t phase = P_CLAIM;
    uint32_t i = 0;
    int32_t s = 0;            // scan position (Alg. 2's id ordering)
    int32_t chunk = -1;       // base of the 16 state bytes held in pq (-1: none)
    int32_t h = 0;            // head of the walk / current node of an absorbed walk
    uint32_t sp = 0;          // stack depth
    uint32_t e0 = 0;          // stack entry 0 (the walk's start), kept in a register
    uint32_t pa = 0;          // state byte of h (in flight)
    uint64_t pb = 0;          // row record of h (in flight)
    ulonglong2 pq = make_ulonglong2(0, 0);
    uint64_t y1 = 0, t = 0, y2 = 0;
    double m2 = 0.0;          // control variate: the sample's pi-walk martingale
    int32_t cv_u = -1;        // control variate: node of the draw whose potential is pending
    long long cv_val = 0;
    unsigned long long acc1 = 0, acc2 = 0;
    unsigned int bad = 0;

    for (;;) {
        if (phase == P_WALK) {
            // Control variate: add the previous draw's potential (its load was
            // issued with that draw's state and row loads).
            if (CV && cv_u >= 0) {
                if ((uint32_t)cv_u < (uint32_t)n) atomicAdd(&p.cv_a1[cv_u], (unsigned long long)cv_val);
                else bad |= LAP_DEV_BAD_INDEX;
                cv_u = -1;
            }
            // One Wilson step per iteration, so walking lanes stay converged.
            // The column entry for draw index 0 (the usual case: the first
            // visit of h) is requested as soon as h's row record arrives,
            // overlapping the state-byte read; it is redone if h was drawn before.
            const int32_t off = row_off(pb);
            const uint32_t deg = row_deg(pb);
            int32_t w = ld_col(col + off + (int64_t)lap::below(lap::philox_r64((uint32_t)h, 0u, i, 0u, key0, key1), deg), keep);
            const uint32_t b = pa;
            if (!b_tree(b, ep)) {
                if (b_path(b, ep)) sp = erase_loop(st, stk, sp, ep, (uint32_t)h, pq, chunk);
                const uint32_t kh = b_k(b, ep);
                if (kh) w = ld_col(col + off + (int64_t)lap::below(lap::philox_r64((uint32_t)h, kh, i, 0u, key0, key1), deg), keep);
                const uint32_t kn = kh + 1u;
                if (kn > kKMax || sp >= cap) {
                    withdraw_sample(st, n, ep, p.rep1, rowinfo, col, CV ? p.cv_h1 : nullptr, p.cv_a1, i, key0, key1);
                    const unsigned int ix = atomicAdd(&p.acc->ovf_count, 1u);
                    if (ix < p.count) p.ovf_ids[ix] = i;
                    phase = P_CLAIM;
                    continue;
                }
                const uint32_t e = (uint32_t)h | (kn << kEntryShift);
                if (sp == 0) e0 = e;
                st_stack(stk + sp, e, keep);
                ++sp;
                st_state(st + h, ep | kBPath | kn);
                pq_set(pq, chunk, (uint32_t)h, ep | kBPath | kn);
                if (kh) atomicAdd(&p.rep1[h], 1ull);
                if (++y1 > limit) { bad |= LAP_DEV_STEP_LIMIT; phase = P_CLAIM; continue; }
                if (CV && p.cv_h1) {
                    cv_u = h;
                    cv_val = p.cv_h1[w];
                }
                h = w;
                pa = ld_state(st + w);
                pb = ld_row(rowinfo, w, keep);
                continue;
            }
            // h is InTree: Alg. 2's retrace adds the loop-erased path on the
            // stack to the tree (draw counts kept, see withdraw_sample).
            if (sp == 1) {
                st_state(st + (e0 & kNodeMask), ep | kBTree | (e0 >> kEntryShift));
                pq_set(pq, chunk, e0 & kNodeMask, ep | kBTree | (e0 >> kEntryShift));
            } else if (sp > 1) {
                commit_path(st, stk, sp, ep, pq, chunk);
            }
            sp = 0;
            ++s;
            phase = P_SCAN;
        }
        if (phase == P_SCAN) {
            // Next start: the first node >= s not InTree, read from the exact
            // copy of the 16 state bytes at `chunk` held in pq.
            if (s < n) {
                const int32_t base = s & ~15;
                if (base != chunk) {
                    pq = *reinterpret_cast<const ulonglong2 *>(st + base);
                    chunk = base;
                    continue;
                }
                uint32_t m = not_tree_mask(pq, ep) & (0xFFFFu << (s - base));
                if (n - base < 16) m &= (1u << (n - base)) - 1u;
                if (m) {
                    s = base + __ffs(m) - 1;
                    h = s;
                    pa = (uint32_t)((((s - base) < 8 ? pq.x : pq.y) >> (8 * ((s - base) & 7))) & 0xFFu);
                    pb = ld_row(rowinfo, h, keep);
                    phase = P_WALK;
                    continue;
                }
                s = base + 16;
                if (s < n) {
                    pq = *reinterpret_cast<const ulonglong2 *>(st + s);
                    chunk = s;
                    continue;
                }
            }
            phase = P_USTART_IMMEDIATE;
        }
        if (phase == P_USTART_IMMEDIATE) {
            // Alg. 2: uniformly sample s in V; walk until v, counting passes.
            t = 0;
            h = (int32_t)lap::below(lap::philox_r64(0u, 0u, i, 1u, key0, key1), (uint64_t)n);
            if (h != v) { atomicAdd(&p.cnt2[h], 1ull); pb = ld_row(rowinfo, h, keep); phase = P_UWALK; continue; }
            phase = P_PISTART_IMMEDIATE;
        }
        if (phase == P_UWALK) {
            ++t;
            const uint64_t r = lap::philox_r64((uint32_t)t, 0u, i, 1u, key0, key1);
            h = ld_col(col + row_off(pb) + (int64_t)lap::below(r, row_deg(pb)), keep);
            if (t > limit) { bad |= LAP_DEV_STEP_LIMIT; phase = P_CLAIM; continue; }
            if (h != v) { atomicAdd(&p.cnt2[h], 1ull); pb = ld_row(rowinfo, h, keep); continue; }
            phase = P_PISTART_IMMEDIATE;
        }
        if (phase == P_PISTART_IMMEDIATE) {
            // Alg. 4: s ~ pi is the head of a uniformly drawn arc.
            y2 = 0;
            m2 = 0.0;
            h = ld_col(col + (int64_t)lap::below(lap::philox_r64(0u, 0u, i, 2u, key0, key1), (uint64_t)p.g.arcs), keep);
            if (h != v) { pb = ld_row(rowinfo, h, keep); phase = P_PIWALK; continue; }
            phase = P_FINISH_IMMEDIATE;
        }
        if (phase == P_PIWALK) {
            ++y2;
            const uint64_t r = lap::philox_r64((uint32_t)y2, 0u, i, 2u, key0, key1);
            const int32_t w = ld_col(col + row_off(pb) + (int64_t)lap::below(r, row_deg(pb)), keep);
            if (CV && p.cv_h2) {
                if ((uint32_t)h >= (uint32_t)n || (uint32_t)w >= (uint32_t)n) {
                    bad |= LAP_DEV_BAD_INDEX;
                    p.acc->pad[0] = ((unsigned long long)(uint32_t)h << 32) | (uint32_t)w;
                    phase = P_CLAIM;
                    continue;
                }
                const long long d = (long long)row_deg(pb), hw = p.cv_h2[w], s2 = p.cv_S2[h];
                atomicAdd(&p.cv_a2[h], (unsigned long long)hw);
                atomicAdd(&p.cv_p2[h], 1ull);
                m2 = __dadd_rn(m2, __ddiv_rn((double)(d * hw - s2), (double)d));
            }
            h = w;
            if (y2 > limit) { bad |= LAP_DEV_STEP_LIMIT; phase = P_CLAIM; continue; }
            if (h != v) { pb = ld_row(rowinfo, h, keep); continue; }
            phase = P_FINISH_IMMEDIATE;
        }
        if (phase == P_FINISH_IMMEDIATE) {
            acc1 += y1;
            acc2 += y2;
            if (p.y1_out) {
                p.y1_out[i - p.first] = y1;
                p.y2_out[i - p.first] = y2;
                if (CV && p.m2_out) p.m2_out[i - p.first] = m2;
            }
            phase = P_CLAIM;
        }
        if (phase == P_CLAIM) {
            if (bad) break;
            const unsigned int q = atomicAdd(&p.acc->claim, 1u);
            if (q >= p.count) break;
            i = p.first + q;
            ep ^= kBEpoch;
            st[v] = (uint8_t)(ep | kBTree);
            s = 0;
            sp = 0;
            y1 = 0;
            chunk = -1;
            phase = P_SCAN;
        }
    }
    p.slot_epoch[slot] = ep ? 1u : 0u;
    if (acc1) atomicAdd(&p.acc->sum_y1, acc1);
    if (acc2) atomicAdd(&p.acc->sum_y2, acc2);
    if (bad) atomicOr(&p.acc->status, bad);
}

}  // namespace

cudaError_t lap_launch_sample_compact(const LapSampleLaunch &p, cudaStream_t st)
{
    if (p.count == 0 || p.slots == 0) return cudaSuccess;
    int block = p.block > 0 ? p.block : lap_pick_block(p.slots, p.num_sms);
    uint64_t grid = (p.slots + block - 1) / block;
    if (p.cv_h1 || p.cv_h2) lewalk_compact_kernel<true><<<(unsigned)grid, block, 0, st>>>(p);
    else lewalk_compact_kernel<false><<<(unsigned)grid, block, 0, st>>>(p);
    return cudaGetLastError();
}
