// LEWalk sampler (hot-path rows a2-a5): for every sample id i,
//   a2  one Wilson LE_v run (Section 3.4; Alg. 2 walk/retrace loops, Alg. 4
//       "walk length" Y1 with loops included),
//   a3  one v-absorbed walk from a uniform start (Alg. 2),
//   a4  one v-absorbed walk from a pi-distributed start (Alg. 4), length Y2,
//   a5  counts folded into per-node uint64 totals and two uint64 sums.
//
// Design.  One lane owns one sample at a time ("slot") and keeps that
// sample's Wilson state in HBM: one 64-bit word per node,
//     bit 63 epoch | bit 62 InTree | bits 32..61 draws k at the node | bits 0..31 Next
// The word carries the draw count k because draw k at node u uses Philox
// counter (u, k, i, 0) (Wilson's stack entry k of u).  The epoch bit flips
// with every sample a slot takes; every node's word is rewritten during every
// sample (each non-root node is visited at least once, the root is written at
// the start), so a word whose epoch differs from the current one reads as
// "not in tree, k = 0" and no per-sample reset pass is needed.
//
// Every non-root node is visited at least once per run, so visits(u) =
// 1 + (repeat visits); only repeats go to the atomic counter (the 1 per
// sample is added analytically at finalize), which cuts atomics to
// Tr((I-P_v)^{-1}) - (n-1) per sample.
//
// The lane runs a flat state machine: each loop iteration consumes the
// loads issued in the previous iteration and issues the next dependent
// load(s), so lanes of a warp in different phases (scan / walk / retrace /
// absorbed walks) stay converged and keep one gather each in flight.  A
// Wilson step costs two dependent rounds: {state[w], row record of w} in
// parallel, then col[row + j].
#include "lap_internal.h"
#include "philox.cuh"

namespace {

constexpr uint64_t kEpoch = 1ull << 63;
constexpr uint64_t kTree = 1ull << 62;
constexpr uint32_t kKMax = 0x3FFFFFFFu;
// Loop-included paths (LapSampleLaunch::paths): after the Wilson run every
// word is InTree; the uniform-start path clears InTree at the nodes it
// leaves and keeps its departure count in the k field, the pi-start path
// marks them with bit 31 (node ids are < 2^31) and keeps its own count there.
constexpr uint64_t kPiMark = 1ull << 31;

enum Phase : uint32_t {
    P_CLAIM = 0,
    P_SCAN,      // pa = state[s], pb = row record of s
    P_STEP,      // pa = state[u], pb = row record of u (u just reached by a walk)
    P_MOVE,      // pb = col entry chosen at u
    P_RETRACE,   // pa = state[u] on the walk's path from s
    P_USTART,
    P_UDRAW,     // pb = row record of u (uniform walk)
    P_UMOVE,     // pb = next node of the uniform walk
    P_PISTART,
    P_PIDRAW,    // pb = row record of u (pi walk)
    P_PIMOVE,    // pb = next node of the pi walk
    P_DONE
};

__device__ __forceinline__ bool is_current(uint64_t w, uint64_t epoch) { return (w & kEpoch) == epoch; }
__device__ __forceinline__ bool in_tree(uint64_t w, uint64_t epoch) { return is_current(w, epoch) && (w & kTree); }
__device__ __forceinline__ uint32_t draws_of(uint64_t w, uint64_t epoch)
{
    return is_current(w, epoch) ? (uint32_t)(w >> 32) & kKMax : 0u;
}
__device__ __forceinline__ uint64_t ld_row(const int2 *rowinfo, int32_t u)
{
    return (uint64_t)__ldg(reinterpret_cast<const unsigned long long *>(rowinfo) + u);
}
__device__ __forceinline__ int32_t row_off(uint64_t r) { return (int32_t)(uint32_t)r; }
__device__ __forceinline__ uint32_t row_deg(uint64_t r) { return (uint32_t)(r >> 32); }

__global__ void __launch_bounds__(256) lewalk_kernel(LapSampleLaunch p)
{
    const uint64_t slot = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (slot >= p.slots) return;
    const int32_t n = p.g.n;
    const int32_t v = p.root;
    const int2 *__restrict__ rowinfo = p.g.rowinfo;
    const int32_t *__restrict__ col = p.g.col;
    unsigned long long *__restrict__ st = reinterpret_cast<unsigned long long *>(p.ws) + slot * (uint64_t)n;
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    const uint64_t limit = p.step_limit;

    uint64_t epoch = p.slot_epoch[slot] ? kEpoch : 0ull;
    uint32_t phase = P_CLAIM;
    uint32_t i = 0;          // sample id
    int32_t s = 0;           // next start node of Alg. 2's ordering (id order)
    int32_t u = 0;           // current node
    uint32_t k = 0;          // draws at u so far
    uint64_t pa = 0, pb = 0; // loaded values consumed in the next iteration
    uint64_t y1 = 0, t = 0, y2 = 0;
    double m2 = 0.0;          // control variate: the sample's pi-walk martingale
    unsigned long long acc1 = 0, acc2 = 0;
    unsigned int bad = 0;
    bool one_done = false;

    while (phase != P_DONE) {
        if (phase == P_MOVE) {
            // Next[u] := RandomNeighbor(u); count the visit; go to w.
            const int32_t w = (int32_t)(uint32_t)pb;
            st[u] = (unsigned long long)(epoch | ((uint64_t)(k + 1u) << 32) | (uint32_t)w);
            if (k) atomicAdd(&p.rep1[u], 1ull);
            if (p.cv_h1) atomicAdd(&p.cv_a1[u], (unsigned long long)p.cv_h1[w]);
            if (k + 1u >= kKMax) bad |= LAP_DEV_K_OVERFLOW;
            ++y1;
            u = w;
            pa = st[u];
            pb = ld_row(rowinfo, u);
            phase = (y1 > limit || bad) ? P_CLAIM : P_STEP;
            if (y1 > limit) bad |= LAP_DEV_STEP_LIMIT;
        } else if (phase == P_STEP || phase == P_SCAN) {
            if (!in_tree(pa, epoch)) {
                // u (or the start s) is off the tree: draw its k-th stack entry.
                if (phase == P_SCAN) u = s;
                k = draws_of(pa, epoch);
                const uint64_t r = lap::philox_r64((uint32_t)u, k, i, 0u, key0, key1);
                pb = (uint64_t)(uint32_t)__ldg(col + row_off(pb) + (int64_t)lap::below(r, row_deg(pb)));
                phase = P_MOVE;
            } else if (phase == P_STEP) {
                // The walk hit the tree: retrace from its start s.
                u = s;
                pa = st[u];
                phase = P_RETRACE;
            } else {
                ++s;
                if (s < n) { pa = st[s]; pb = ld_row(rowinfo, s); }
                else phase = P_USTART;
            }
        } else if (phase == P_RETRACE) {
            if (!in_tree(pa, epoch)) {
                st[u] = (unsigned long long)(pa | kTree);
                u = (int32_t)(uint32_t)pa;
                pa = st[u];
            } else {
                ++s;
                if (s < n) { pa = st[s]; pb = ld_row(rowinfo, s); phase = P_SCAN; }
                else phase = P_USTART;
            }
        } else if (phase == P_UDRAW) {
            ++t;
            uint64_t r;
            if (p.paths) {
                // Departure j from u takes u's stack entry j (draw (u, j, i, 0)).
                const uint32_t j = (pa & kTree) ? 0u : (uint32_t)(pa >> 32) & kKMax;
                r = lap::philox_r64((uint32_t)u, j, i, 0u, key0, key1);
                st[u] = (unsigned long long)(epoch | ((uint64_t)(j + 1u) << 32) | (pa & 0xFFFFFFFFull));
                atomicAdd(&p.cnt2[u], 1ull);
            } else {
                r = lap::philox_r64((uint32_t)t, 0u, i, 1u, key0, key1);
            }
            pb = (uint64_t)(uint32_t)__ldg(col + row_off(pb) + (int64_t)lap::below(r, row_deg(pb)));
            phase = P_UMOVE;
            if (t > limit) { bad |= LAP_DEV_STEP_LIMIT; phase = P_CLAIM; }
        } else if (phase == P_UMOVE) {
            u = (int32_t)(uint32_t)pb;
            if (u == v) phase = P_PISTART;
            else {
                if (p.paths) pa = st[u];
                else atomicAdd(&p.cnt2[u], 1ull);
                pb = ld_row(rowinfo, u);
                phase = P_UDRAW;
            }
        } else if (phase == P_PIDRAW) {
            ++y2;
            uint64_t r;
            if (p.paths) {
                const uint32_t j = (pa & kPiMark) ? (uint32_t)(pa >> 32) & kKMax : 0u;
                r = lap::philox_r64((uint32_t)u, j, i, 0u, key0, key1);
                st[u] = (unsigned long long)(epoch | (pa & kTree) | ((uint64_t)(j + 1u) << 32) | kPiMark |
                                             (pa & 0x7FFFFFFFull));
            } else {
                r = lap::philox_r64((uint32_t)y2, 0u, i, 2u, key0, key1);
            }
            const int32_t w = __ldg(col + row_off(pb) + (int64_t)lap::below(r, row_deg(pb)));
            if (p.cv_h2) {
                const long long d = (long long)row_deg(pb), hw = p.cv_h2[w], s2 = p.cv_S2[u];
                atomicAdd(&p.cv_a2[u], (unsigned long long)hw);
                atomicAdd(&p.cv_p2[u], 1ull);
                m2 = __dadd_rn(m2, __ddiv_rn((double)(d * hw - s2), (double)d));
            }
            pb = (uint64_t)(uint32_t)w;
            phase = P_PIMOVE;
            if (y2 > limit) { bad |= LAP_DEV_STEP_LIMIT; phase = P_CLAIM; }
        } else if (phase == P_PIMOVE) {
            u = (int32_t)(uint32_t)pb;
            if (u == v) {
                acc1 += y1;
                acc2 += y2;
                if (p.y1_out) {
                    const uint32_t ix = i - (p.ids ? p.trace_base : p.first);
                    p.y1_out[ix] = y1;
                    p.y2_out[ix] = y2;
                    if (p.m2_out) p.m2_out[ix] = m2;
                }
                phase = P_CLAIM;
            }
            else {
                if (p.paths) pa = st[u];
                pb = ld_row(rowinfo, u);
                phase = P_PIDRAW;
            }
        } else if (phase == P_USTART) {
            if (p.flags & LAP_SAMPLE_WILSON_ONLY) {
                acc1 += y1;
                phase = P_CLAIM;
                continue;
            }
            // Alg. 2: uniformly sample s in V (or take the fixed start of a
            // single-source row); walk until v, counting passes.
            t = 0;
            u = p.ustart ? (int32_t)(p.ustart - 1u)
                         : (int32_t)lap::below(lap::philox_r64(0u, 0u, i, 1u, key0, key1), (uint64_t)n);
            if (u == v) phase = P_PISTART;
            else {
                if (p.paths) pa = st[u];
                else atomicAdd(&p.cnt2[u], 1ull);
                pb = ld_row(rowinfo, u);
                phase = P_UDRAW;
            }
        } else if (phase == P_PISTART) {
            // Alg. 4: s ~ pi is the head of a uniformly drawn arc.
            y2 = 0;
            m2 = 0.0;
            const uint64_t r = lap::philox_r64(0u, 0u, i, 2u, key0, key1);
            pb = (uint64_t)(uint32_t)__ldg(col + (int64_t)lap::below(r, (uint64_t)p.g.arcs));
            phase = P_PIMOVE;
        } else {  // P_CLAIM
            if (bad) { phase = P_DONE; break; }
            if (p.flags & LAP_SAMPLE_ONE_PER_LANE) {
                if (one_done || slot >= p.count) { phase = P_DONE; break; }
                one_done = true;
                i = p.first + (uint32_t)slot;
            } else {
                const unsigned int q = atomicAdd(&p.acc->claim, 1u);
                if (q >= p.count) { phase = P_DONE; break; }
                i = p.ids ? p.ids[q] : p.first + q;
            }
            epoch ^= kEpoch;
            st[v] = (unsigned long long)(epoch | kTree);
            s = 0;
            y1 = 0;
            pa = st[0];
            pb = ld_row(rowinfo, 0);
            phase = P_SCAN;
        }
    }
    p.slot_epoch[slot] = epoch ? 1u : 0u;
    if (acc1) atomicAdd(&p.acc->sum_y1, acc1);
    if (acc2) atomicAdd(&p.acc->sum_y2, acc2);
    if (bad) atomicOr(&p.acc->status, bad);
}

}  // namespace

cudaError_t lap_launch_sample(const LapSampleLaunch &p, cudaStream_t st)
{
    if (p.count == 0 || p.slots == 0) return cudaSuccess;
    int block = p.block > 0 ? p.block : lap_pick_block(p.slots, p.num_sms);
    uint64_t lanes = p.slots;
    uint64_t grid = (lanes + block - 1) / block;
    lewalk_kernel<<<(unsigned)grid, block, 0, st>>>(p);
    return cudaGetLastError();
}
