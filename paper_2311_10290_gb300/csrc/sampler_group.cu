// Several-walkers LEWalk sampler ("kernel 3"): W lanes of one warp run one
// sample's Wilson LE_v run together, then two of them run the sample's
// uniform-start and pi-start v-absorbed walks (Alg. 2 and Alg. 4).  The
// counts are those of the sequential run, bit for bit.
//
// Why it is exact.  In the stack representation of Section 3.4 (Fig. 1),
// node u's j-th draw is the j-th entry of u's stack, here the Philox draw
// (u, j, i, 0); Wilson's run pops cycles of stack tops, and the set of popped
// cycles -- hence each node's number of draws (its visits) and the tree --
// does not depend on the order in which cycles are found.  The walkers follow
// the concurrent popping protocol:
//   - a walker owns the nodes of its loop-erased path; at its head u it takes
//     u's pending arrow if an aborted walker left one (no new draw), else
//     draws u's next stack entry (a visit of u);
//   - the arrow's target w is claimed with a compare-and-swap if free; if w
//     is in the tree the path joins the tree; if w is on the walker's own
//     path the closed cycle is popped (its nodes' arrows are consumed);
//   - if w is on another walker's path, a lower-numbered walker waits and
//     tries again, a higher-numbered one aborts: its nodes are released with
//     their current arrows pending (the arrow of a node is always its last
//     draw, k - 1), so no stack entry is lost.
// Waits go from lower- to higher-numbered walkers only, so they cannot form a
// cycle; the highest-numbered active walker always progresses.
//
// State per node and sample in flight, 16 bits, cleared at each sample start:
//   bit 15 InTree | bit 14 pending | owner (walker + 1, 0 = free; 4 bits for up
//   to 8 walkers, 5 for 16) | draws k (the remaining 10 or 9 bits)
// A path node's arrow is never stored: it is draw k - 1.  A walker keeps its
// path on a private stack (entries node | k << 22), the head in a register.
// Start nodes come from a per-sample chunk cursor (32 nodes per chunk); past
// the last chunk the cursor wraps around (sweeps pick up nodes released by
// aborts and popped cycles behind it) until every node is in the tree.
//
// A sample that does not fit (a node drawn 1023 (511) times, a path longer than the
// walker's stack, or a walker without progress for kStallNs) is withdrawn
// exactly as in the 1-byte kernel: the group subtracts k - 1 for every node
// (and, with the control variate, the potentials of all k draws) and lists
// the id for a re-run with the 8-byte kernel.
//
// Control variate (CV): each Wilson draw of u with target w adds h1[w] to
// A1[u] (once per draw: a pending arrow taken again adds nothing), and the
// pi-start walk adds h2[w] to A2[u], 1 to P2[u] and (d_u h2[w] - S2[u]) / d_u
// to the sample's M2, as in the other samplers.
//
// Loop-included paths (PATHS): the two absorbed walks take the sample's own
// stacks (departure j from u follows u's stack entry j, the Philox draw
// (u, j, i, 0)), counting departures per node in one byte per walk (a region
// of 2 bytes per node after the state words).  A node left 255 times by one
// walk withdraws the sample; the group then also subtracts the walks'
// departures (cnt2, and with the CV the pi walk's A2 and P2 terms).
#include "lap_internal.h"
#include "philox.cuh"

namespace {

constexpr uint32_t kGTree = 0x8000u, kGPend = 0x4000u;

// Owner and draw-count fields of the 16-bit word: 4 owner bits and 10 count
// bits for up to 8 walkers, 5 and 9 for 16.
template <int W>
struct GWord {
    static constexpr uint32_t own_bits = W <= 8 ? 4u : 5u;
    static constexpr uint32_t shift = 14u - own_bits;
    static constexpr uint32_t own = ((1u << own_bits) - 1u) << shift;
    static constexpr uint32_t k = (1u << shift) - 1u;
    static constexpr uint32_t kmax = k;                 // a node drawn this often withdraws the sample
};
constexpr int kNodeBits = 22;
constexpr uint32_t kGNode = (1u << kNodeBits) - 1u;
constexpr uint32_t kChunk = 32;                                   // nodes per scan chunk (64 bytes)
constexpr unsigned long long kStallNs = 4000000000ull;            // 4 s without progress: withdraw
constexpr unsigned int kWithdraw = 1u;

struct GroupCtl {              // first 64 bytes of a slot
    unsigned int cursor;       // scan chunks claimed so far (grows past the chunk count: sweeps)
    unsigned int tree;         // nodes in the tree, the root included
    unsigned int status;       // kWithdraw
    unsigned int pad0;
    unsigned long long y1;     // the walkers' draws
    unsigned long long pad[5];
};

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t ld_word(const uint16_t *a)
{
    uint16_t v;
    asm volatile("ld.global.cg.u16 %0, [%1];" : "=h"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_word(uint16_t *a, uint32_t v)
{
    asm volatile("st.global.cg.u16 [%0], %1;" ::"l"(a), "h"((uint16_t)v) : "memory");
}
__device__ __forceinline__ uint4 ld_chunk4(const uint16_t *a)
{
    uint4 v;
    asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ unsigned int ld_u32(const unsigned int *a)
{
    unsigned int v;
    asm volatile("ld.global.cg.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_u64(const unsigned long long *a)
{
    unsigned long long v;
    asm volatile("ld.global.cg.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t cas_word(uint16_t *a, uint32_t expect, uint32_t val)
{
    return atomicCAS(reinterpret_cast<unsigned short int *>(a), (unsigned short int)expect, (unsigned short int)val);
}
template <int W>
__device__ __forceinline__ bool w_free(uint32_t w) { return (w & (kGTree | GWord<W>::own)) == 0u; }
template <int W>
__device__ __forceinline__ uint32_t w_owner(uint32_t w) { return (w & GWord<W>::own) >> GWord<W>::shift; }

// Bit b set when word b of the 32 words (two per 32-bit lane of the four
// vectors) is neither in the tree nor owned.
template <int W>
__device__ __forceinline__ uint32_t free_mask2(uint32_t x)
{
    const uint32_t e = __vcmpeq2(x & ((kGTree | GWord<W>::own) * 0x00010001u), 0u);   // 0xFFFF per free half
    return (e & 1u) | ((e >> 15) & 2u);
}
template <int W>
__device__ __forceinline__ uint32_t free_mask(uint4 a, uint4 b, uint4 c, uint4 d)
{
    const uint32_t q[16] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w, d.x, d.y, d.z, d.w};
    uint32_t m = 0;
#pragma unroll
    for (int t = 0; t < 16; ++t) m |= free_mask2<W>(q[t]) << (2 * t);
    return m;
}

// The graph (row records, columns) should stay in L2 while the state words
// stream through it.
__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t ld_row(const int2 *rowinfo, int32_t u, uint64_t pol)
{
    uint64_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(rowinfo + u), "l"(pol));
    return v;
}
__device__ __forceinline__ int32_t ld_col(const int32_t *a, uint64_t pol)
{
    int32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ long long ld_pot(const long long *a)
{
    long long v;
    asm volatile("ld.global.nc.s64 %0, [%1];" : "=l"(v) : "l"(a));
    return v;
}
// Target of draw k at node u (row record r of u), sample i.
__device__ __forceinline__ int32_t arrow_of(const int32_t *col, uint64_t r, uint32_t u, uint32_t k, uint32_t i,
                                            uint32_t key0, uint32_t key1, uint64_t pol)
{
    return ld_col(col + (int64_t)(int32_t)(uint32_t)r + (int64_t)lap::below(lap::philox_r64(u, k, i, 0u, key0, key1),
                                                                             (uint32_t)(r >> 32)), pol);
}

enum : uint32_t { G_SCAN = 0, G_STEP, G_MOVE, G_DONE };

template <int W, bool CV, bool PATHS>
__global__ void __launch_bounds__(256, 5) lewalk_group_kernel(LapSampleLaunch p)
{
    static_assert(W == 2 || W == 4 || W == 8 || W == 16, "walkers per sample");
    using L = GWord<W>;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t gbase = lane & ~(uint32_t)(W - 1);
    const unsigned gmask = ((1u << W) - 1u) << gbase;
    const uint32_t j = lane - gbase;                    // walker index in the group
    const uint32_t mine = (j + 1u) << L::shift;         // owner field of this walker
    const uint64_t slot = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) / W;
    if (slot >= p.slots) return;                        // uniform over the group
    const int32_t n = p.g.n;
    const int32_t v = p.root;
    const int2 *__restrict__ rowinfo = p.g.rowinfo;
    const int32_t *__restrict__ col = p.g.col;
    uint8_t *base = reinterpret_cast<uint8_t *>(p.ws) + slot * p.slot_bytes;
    GroupCtl *ctl = reinterpret_cast<GroupCtl *>(base);
    uint16_t *st = reinterpret_cast<uint16_t *>(base + 64);
    uint8_t *pc = base + 64 + 2ull * p.n_pad;           // PATHS: departures, 2 bytes per node
    const uint32_t cap = p.stack_cap;                   // entries per walker, a multiple of 4
    uint32_t *stk = reinterpret_cast<uint32_t *>(base + 64 + (PATHS ? 4ull : 2ull) * p.n_pad) + (uint64_t)j * cap;
    const uint32_t nchunks = (uint32_t)((n + (int32_t)kChunk - 1) / (int32_t)kChunk);   // chunks holding nodes
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    const uint64_t limit = p.step_limit;
    const uint64_t keep = policy_evict_last();
    unsigned long long acc1 = 0, acc2 = 0;
    unsigned int bad = 0;

    for (;;) {
        unsigned int q = 0;
        if (j == 0) q = atomicAdd(&p.acc->claim, 1u);
        q = __shfl_sync(gmask, q, (int)gbase);
        if (q >= p.count) break;
        const uint32_t i = p.first + q;

        // Clear the slot's state and control block; the root starts in the tree.
        {
            uint4 *s4 = reinterpret_cast<uint4 *>(st);
            const uint64_t n4 = (PATHS ? 4ull : 2ull) * p.n_pad / 16u;    // state words and departure bytes
            for (uint64_t x = j; x < n4; x += W) s4[x] = make_uint4(0u, 0u, 0u, 0u);
            if (j == 0) {
                uint4 *c4 = reinterpret_cast<uint4 *>(ctl);
                for (int x = 0; x < 4; ++x) c4[x] = make_uint4(0u, 0u, 0u, 0u);
            }
            __threadfence();
            __syncwarp(gmask);
            if (j == 0) {
                st[v] = (uint16_t)kGTree;
                ctl->tree = 1u;
            }
            __threadfence();
            __syncwarp(gmask);
        }

        uint32_t phase = G_SCAN;
        uint32_t cbase = 0, cmask = 0;       // current scan chunk and its candidate starts
        int32_t h = 0;                       // head of the walker's path
        uint32_t hk = 0;                     // draws of the head
        bool hpend = false;                  // the head's arrow is pending (taken without a draw)
        uint64_t hrow = 0;                   // row record of the head
        uint32_t sp = 0;                     // path length (stack entries 0 .. sp-2 in memory, the head in `top`)
        uint32_t top = 0;
        int32_t w = 0;                       // target of the head's arrow (G_MOVE)
        uint32_t ew = 0;                     // expected word of w for the claim (all ones: read it first)
        uint64_t y1 = 0;
        uint32_t committed = 0;              // nodes this walker added to the tree, not yet in ctl->tree
        uint32_t iter = 0;
        bool cvp = false;                    // CV: the head's new draw still owes h1[w] to A1[h]
        unsigned long long tprog = 0;        // last progress (set when a wait or an idle sweep begins)
        bool waiting = false;
        bool withdraw = false;

        while (phase != G_DONE) {
            if (phase == G_SCAN) {
                if (cmask == 0u) {
                    // The tree count is published once per chunk: the sample ends
                    // when every walker's additions are in (no walker that still
                    // holds a path or unpublished nodes can see the full count).
                    if (committed) {
                        atomicAdd(&ctl->tree, committed);
                        committed = 0;
                    }
                    if (ld_u32(&ctl->tree) >= (unsigned)n || ld_u32(&ctl->status)) { phase = G_DONE; break; }
                    const unsigned int c = atomicAdd(&ctl->cursor, 1u);
                    const uint32_t ch = c % nchunks;
                    cbase = ch * kChunk;
                    const uint16_t *cp = st + cbase;
                    const uint4 a = ld_chunk4(cp), b = ld_chunk4(cp + 8), cc = ld_chunk4(cp + 16), d = ld_chunk4(cp + 24);
                    cmask = free_mask<W>(a, b, cc, d);
                    // The last chunk holds 1..31 nodes: cbase < n <= cbase + 32.
                    if (cbase + kChunk > (uint32_t)n) cmask &= (1u << ((uint32_t)n - cbase)) - 1u;
                    if (c >= nchunks && cmask == 0u) {
                        // An idle sweep: the remaining nodes are on other walkers' paths.
                        if (!waiting) { waiting = true; tprog = now_ns(); }
                        else if (now_ns() - tprog > kStallNs) { withdraw = true; phase = G_DONE; break; }
                        __nanosleep(200);
                    }
                    continue;
                }
                const int32_t s = (int32_t)(cbase + (uint32_t)__ffs(cmask) - 1u);
                cmask &= cmask - 1u;
                // Claim the start: most nodes are untouched (word 0) on the first pass.
                uint32_t expect = 0u;
                uint32_t old = cas_word(st + s, expect, mine);
                const uint64_t row = ld_row(rowinfo, s, keep);
                for (int t = 0; t < 8 && old != expect && w_free<W>(old); ++t) {
                    expect = old;
                    old = cas_word(st + s, expect, expect | mine);
                }
                if (old != expect) continue;           // in the tree, or taken by another walker
                waiting = false;
                h = s;
                hk = old & L::k;
                hpend = (old & kGPend) != 0u;
                hrow = row;
                sp = 1;
                top = (uint32_t)s | (hk << kNodeBits);
                phase = G_STEP;
                continue;
            }
            if (phase == G_STEP) {
                // Checked before a draw, so that every counted draw reaches G_MOVE
                // (where its control-variate term is added).
                if (((++iter) & 255u) == 0u && ld_u32(&ctl->status)) { phase = G_DONE; break; }
                // Take the head's arrow: its pending one, or its next stack entry.
                uint32_t kd;
                if (hpend) {
                    kd = hk - 1u;
                    hpend = false;
                } else {
                    if (hk >= L::kmax) { withdraw = true; phase = G_DONE; break; }   // top holds hk
                    kd = hk;
                    ++hk;
                    ++y1;
                    if (kd) atomicAdd(&p.rep1[h], 1ull);
                    // The head's word is written when the path commits, aborts or
                    // pops (or the sample is withdrawn): until then only its owner
                    // reads its draw count, from the path entry.
                    top = (uint32_t)h | (hk << kNodeBits);
                    if (y1 > limit) { bad |= LAP_DEV_STEP_LIMIT; withdraw = true; phase = G_DONE; break; }
                    cvp = CV && p.cv_h1;
                }
                top = (uint32_t)h | (hk << kNodeBits);
                w = arrow_of(col, hrow, (uint32_t)h, kd, i, key0, key1, keep);
                ew = 0xFFFFFFFFu;
                phase = G_MOVE;
                // fall through to the claim in the same iteration
            }
            if (phase == G_MOVE) {
                // Read w's word; only a free node needs the compare-and-swap
                // that claims it (InTree is final, so a plain read of it is
                // conclusive; most steps end in the tree).
                const uint64_t row = ld_row(rowinfo, w, keep);
                long long hv = 0;
                if (CV && cvp) hv = ld_pot(p.cv_h1 + w);     // issued with the row and word reads
                uint32_t old;
                bool claimed = false;
                if (ew == 0xFFFFFFFFu) {
                    old = ld_word(st + w);
                    if (CV && cvp) {
                        atomicAdd(&p.cv_a1[h], (unsigned long long)hv);
                        cvp = false;
                    }
                    if (w_free<W>(old)) {
                        ew = old;
                        old = cas_word(st + w, ew, ew | mine);
                        claimed = old == ew;
                    }
                } else {
                    old = cas_word(st + w, ew, ew | mine);
                    claimed = old == ew;
                }
                for (int t = 0; t < 8 && !claimed && w_free<W>(old); ++t) {
                    ew = old;
                    old = cas_word(st + w, ew, ew | mine);
                    claimed = old == ew;
                }
                if (claimed) {
                    // w joins the path as its new head.
                    if (sp >= cap) { withdraw = true; phase = G_DONE; break; }
                    stk[sp - 1] = top;
                    ++sp;
                    h = w;
                    hk = old & L::k;
                    hpend = (old & kGPend) != 0u;
                    hrow = row;
                    top = (uint32_t)w | (hk << kNodeBits);
                    waiting = false;
                    phase = G_STEP;
                    continue;
                }
                if (old & kGTree) {
                    // The loop-erased path joins the tree (Alg. 2's retrace).
                    st_word(st + (top & kGNode), kGTree | (top >> kNodeBits));
                    for (uint32_t x = 0; x + 1u < sp; ++x) {
                        const uint32_t e = stk[x];
                        st_word(st + (e & kGNode), kGTree | (e >> kNodeBits));
                    }
                    // No fence: another walker that still reads such a node as
                    // owned waits or aborts, both exact.
                    committed += sp;
                    sp = 0;
                    waiting = false;
                    phase = G_SCAN;
                    continue;
                }
                const uint32_t o = w_owner<W>(old);
                if (o == j + 1u) {
                    // A cycle of stack tops closed at w: pop it; w draws again.
                    st_word(st + h, hk);
                    uint32_t x = sp - 1u;            // entries 0 .. sp-2 are in memory
                    uint32_t e = 0;
                    for (;;) {
                        if (x == 0u) { bad |= LAP_DEV_BAD_INDEX; withdraw = true; break; }
                        e = stk[--x];
                        if ((int32_t)(e & kGNode) == w) break;
                        st_word(st + (e & kGNode), e >> kNodeBits);
                    }
                    if (withdraw) { phase = G_DONE; break; }
                    sp = x + 1u;
                    top = e;
                    h = w;
                    hk = e >> kNodeBits;
                    hpend = false;
                    hrow = row;
                    waiting = false;
                    phase = G_STEP;
                    continue;
                }
                if (j + 1u > o) {
                    // Abort: every node of the path keeps its arrow as pending.
                    st_word(st + (top & kGNode), kGPend | (top >> kNodeBits));
                    for (uint32_t x = 0; x + 1u < sp; ++x) {
                        const uint32_t e = stk[x];
                        st_word(st + (e & kGNode), kGPend | (e >> kNodeBits));
                    }
                    sp = 0;
                    waiting = false;
                    phase = G_SCAN;
                    continue;
                }
                // Wait for the higher-numbered walker; try the same arrow again.
                if (!waiting) { waiting = true; tprog = now_ns(); }
                else if (now_ns() - tprog > kStallNs) { withdraw = true; phase = G_DONE; break; }
                if (ld_u32(&ctl->status)) { phase = G_DONE; break; }
                ew = 0xFFFFFFFFu;
                __nanosleep(100);
                continue;
            }
        }

        if (withdraw) atomicOr(&ctl->status, kWithdraw);
        // A walker stopped with a path (the sample is being withdrawn) writes
        // its nodes' draw counts, so that the subtraction below sees them.
        if (sp > 0) {
            st_word(st + (top & kGNode), top >> kNodeBits);
            for (uint32_t x = 0; x + 1u < sp; ++x) {
                const uint32_t e = stk[x];
                st_word(st + (e & kGNode), e >> kNodeBits);
            }
        }
        atomicAdd(&ctl->y1, (unsigned long long)y1);
        __threadfence();
        __syncwarp(gmask);
        // One lane reads the status and the group takes its value: with PATHS a
        // walk below may set kWithdraw while a slower walker of the group has
        // not read it yet, and every walker must take the same branch (they
        // meet at warp barriers).
        bool wdrawn = __shfl_sync(gmask, (int)(j == 0 && (ld_u32(&ctl->status) & kWithdraw) != 0u), (int)gbase) != 0;
        uint64_t y2 = 0;
        double m2 = 0.0;
        if (!wdrawn) {
            if (j == 0) {
                // Alg. 2: the v-absorbed walk from a uniform start (or the fixed
                // start of a single-source row), counting passes; with PATHS,
                // the loop-included path on the sample's stacks.
                uint64_t t = 0;
                int32_t u = p.ustart ? (int32_t)(p.ustart - 1u)
                                     : (int32_t)lap::below(lap::philox_r64(0u, 0u, i, 1u, key0, key1), (uint64_t)n);
                if (!PATHS) {
                    while (u != v) {
                        atomicAdd(&p.cnt2[u], 1ull);
                        if (++t > limit) { bad |= LAP_DEV_STEP_LIMIT; break; }
                        const uint64_t r = ld_row(rowinfo, u, keep);
                        u = ld_col(col + (int64_t)(int32_t)(uint32_t)r +
                                   (int64_t)lap::below(lap::philox_r64((uint32_t)t, 0u, i, 1u, key0, key1), (uint32_t)(r >> 32)), keep);
                    }
                } else {
                    while (u != v) {
                        if (++t > limit) { bad |= LAP_DEV_STEP_LIMIT; break; }
                        const uint32_t jd = pc[2 * (int64_t)u];
                        if (jd == 255u) { atomicOr(&ctl->status, kWithdraw); break; }
                        const uint64_t r = ld_row(rowinfo, u, keep);
                        const int32_t x = arrow_of(col, r, (uint32_t)u, jd, i, key0, key1, keep);
                        pc[2 * (int64_t)u] = (uint8_t)(jd + 1u);
                        atomicAdd(&p.cnt2[u], 1ull);
                        u = x;
                    }
                }
            }
            if (j == 1u) {
                // Alg. 4: the v-absorbed walk from s ~ pi (the head of a uniform
                // arc); Y2 = its length.  With PATHS, the loop-included path.
                int32_t u = ld_col(col + (int64_t)lap::below(lap::philox_r64(0u, 0u, i, 2u, key0, key1), (uint64_t)p.g.arcs), keep);
                while (u != v) {
                    if (++y2 > limit) { bad |= LAP_DEV_STEP_LIMIT; break; }
                    const uint64_t r = ld_row(rowinfo, u, keep);
                    int32_t x;
                    if (PATHS) {
                        const uint32_t jd = pc[2 * (int64_t)u + 1];
                        if (jd == 255u) { atomicOr(&ctl->status, kWithdraw); break; }
                        x = arrow_of(col, r, (uint32_t)u, jd, i, key0, key1, keep);
                        pc[2 * (int64_t)u + 1] = (uint8_t)(jd + 1u);
                    } else {
                        x = ld_col(col + (int64_t)(int32_t)(uint32_t)r +
                                   (int64_t)lap::below(lap::philox_r64((uint32_t)y2, 0u, i, 2u, key0, key1), (uint32_t)(r >> 32)), keep);
                    }
                    if (CV && p.cv_h2) {
                        const long long d = (long long)(r >> 32), hx = ld_pot(p.cv_h2 + x), s2 = ld_pot(p.cv_S2 + u);
                        atomicAdd(&p.cv_a2[u], (unsigned long long)hx);
                        atomicAdd(&p.cv_p2[u], 1ull);
                        m2 = __dadd_rn(m2, __ddiv_rn((double)(d * hx - s2), (double)d));
                    }
                    u = x;
                }
            }
            if (PATHS) {
                // A walk that met a node's 255th departure withdraws the sample.
                __threadfence();
                __syncwarp(gmask);
                wdrawn = __shfl_sync(gmask, (int)(j == 0 && (ld_u32(&ctl->status) & kWithdraw) != 0u), (int)gbase) != 0;
            }
        }
        if (wdrawn) {
            // Withdraw the sample: subtract the repeat visits counted so far
            // (and the control-variate and path terms added so far).
            for (int32_t x = (int32_t)j; x < n; x += W) {
                const uint32_t k = ld_word(st + x) & L::k;
                if (k >= 2u) atomicAdd(&p.rep1[x], (unsigned long long)(-(long long)(k - 1u)));
                if (CV && p.cv_h1 && k) {
                    // The potentials of all k draws, added to A1[x] one per draw.
                    const uint64_t r = ld_row(rowinfo, x, keep);
                    long long sub = 0;
                    for (uint32_t d = 0; d < k; ++d) sub += ld_pot(p.cv_h1 + arrow_of(col, r, (uint32_t)x, d, i, key0, key1, keep));
                    atomicAdd(&p.cv_a1[x], (unsigned long long)(-sub));
                }
                if (PATHS) {
                    const uint32_t cu = pc[2 * (int64_t)x], cp = pc[2 * (int64_t)x + 1];
                    if (cu) atomicAdd(&p.cnt2[x], (unsigned long long)(-(long long)cu));
                    if (CV && p.cv_h2 && cp) {
                        const uint64_t r = ld_row(rowinfo, x, keep);
                        long long sub = 0;
                        for (uint32_t d = 0; d < cp; ++d) sub += ld_pot(p.cv_h2 + arrow_of(col, r, (uint32_t)x, d, i, key0, key1, keep));
                        atomicAdd(&p.cv_a2[x], (unsigned long long)(-sub));
                        atomicAdd(&p.cv_p2[x], (unsigned long long)(-(long long)cp));
                    }
                }
            }
            if (j == 0) {
                const unsigned int ix = atomicAdd(&p.acc->ovf_count, 1u);
                if (ix < p.count) p.ovf_ids[ix] = i;
            }
        } else {
            if (j == 0) {
                const unsigned long long sy1 = ld_u64(&ctl->y1);
                acc1 += sy1;
                if (p.y1_out) p.y1_out[i - p.first] = sy1;
            }
            if (j == 1u) {
                acc2 += y2;
                if (p.y2_out) p.y2_out[i - p.first] = y2;
                if (CV && p.m2_out) p.m2_out[i - p.first] = m2;
            }
        }
        __syncwarp(gmask);
    }
    if (acc1) atomicAdd(&p.acc->sum_y1, acc1);
    if (acc2) atomicAdd(&p.acc->sum_y2, acc2);
    if (bad) atomicOr(&p.acc->status, bad);
}

template <int W>
void launch_group(const LapSampleLaunch &p, bool cv, uint64_t grid, int block, cudaStream_t st)
{
    if (p.paths) {
        if (cv) lewalk_group_kernel<W, true, true><<<(unsigned)grid, block, 0, st>>>(p);
        else lewalk_group_kernel<W, false, true><<<(unsigned)grid, block, 0, st>>>(p);
    } else {
        if (cv) lewalk_group_kernel<W, true, false><<<(unsigned)grid, block, 0, st>>>(p);
        else lewalk_group_kernel<W, false, false><<<(unsigned)grid, block, 0, st>>>(p);
    }
}

}  // namespace

cudaError_t lap_launch_sample_group(const LapSampleLaunch &p, int walkers, cudaStream_t st)
{
    if (p.count == 0 || p.slots == 0) return cudaSuccess;
    const uint64_t lanes = p.slots * (uint64_t)walkers;
    const int block = 256;
    const uint64_t grid = (lanes + block - 1) / block;
    const bool cv = p.cv_h1 || p.cv_h2;
    if (walkers == 2) launch_group<2>(p, cv, grid, block, st);
    else if (walkers == 4) launch_group<4>(p, cv, grid, block, st);
    else if (walkers == 8) launch_group<8>(p, cv, grid, block, st);
    else if (walkers == 16) launch_group<16>(p, cv, grid, block, st);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}
