// Per-lane Wilson state of the compact samplers (sampler_compact.cu for one
// graph, sampler_batch.cu for a batch of graphs): one byte per node and
// sample in flight plus a per-lane stack holding the loop-erased path.
//
// Per node and sample one byte:   bit 7 epoch | bit 6 InTree | bit 5 OnPath | bits 0..4 draws k
// Stack entries: node | k << 27 (k as in the byte).
//
// Draw counts k <= 30 live in the byte.  From the 31st draw at a node on, the
// byte holds kKSat and the count lives in a per-lane open-addressing table
// after the path stack: 2^tbl_log2 entries {key : 32 | tag : 8 | k : 24}, the
// key being the node and the kind of count (Wilson draws, or departures of
// one of the loop-included paths when the absorbed walks are taken on the
// sample's own stacks).  Each sample of a lane has its own tag (1..255), so
// entries of earlier samples read as empty and the table is cleared only when
// the tag wraps (and at the lane's first sample).  A sample that needs more
// entries than a probe run of kTblProbes finds, more than kKMax draws at a
// node, or a longer path than the stack holds is withdrawn.
#pragma once

#include "lap_internal.h"
#include "philox.cuh"

namespace lap_compact {

// Functions are static: every translation unit keeps its own copy.

constexpr uint32_t kBEpoch = 0x80u, kBTree = 0x40u, kBPath = 0x20u, kBK = 0x1Fu;
constexpr uint32_t kKSat = 31u;                 // byte value: "count in the table"
constexpr uint32_t kKMax = (1u << 24) - 1u;       // draws at one node in one sample
constexpr uint32_t kTblProbes = 32u;
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
static __device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// State bytes: default L2 priority (a sector read at one step is written at
// the next step and again at the retrace, so it should stay in L2 meanwhile;
// evicting it early turns those writes into partial-sector fills), no L1
// allocation (no reuse within a lane at L1 time scales).
static __device__ __forceinline__ uint32_t ld_state(const uint8_t *a)
{
    uint16_t v;
    asm volatile("ld.global.L1::no_allocate.u8 %0, [%1];" : "=h"(v) : "l"(a) : "memory");
    return v;
}
static __device__ __forceinline__ void st_state(uint8_t *a, uint32_t v)
{
    asm volatile("st.global.L1::no_allocate.u8 [%0], %1;" ::"l"(a), "h"((uint16_t)v) : "memory");
}
// Path-stack entries: kept in L2 with the graph (they are re-read at the retrace).
static __device__ __forceinline__ void st_stack(uint32_t *a, uint32_t v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(pol) : "memory");
}
static __device__ __forceinline__ int32_t ld_col(const int32_t *a, uint64_t pol)
{
    int32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}
static __device__ __forceinline__ uint64_t ld_row(const int2 *rowinfo, int32_t u, uint64_t pol)
{
    uint64_t v;
    asm volatile("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(rowinfo + u), "l"(pol));
    return v;
}

static __device__ __forceinline__ bool b_current(uint32_t b, uint32_t ep) { return (b & kBEpoch) == ep; }
static __device__ __forceinline__ bool b_tree(uint32_t b, uint32_t ep) { return b_current(b, ep) && (b & kBTree); }
static __device__ __forceinline__ bool b_path(uint32_t b, uint32_t ep) { return b_current(b, ep) && (b & kBPath); }
static __device__ __forceinline__ uint32_t b_k(uint32_t b, uint32_t ep) { return b_current(b, ep) ? (b & kBK) : 0u; }
static __device__ __forceinline__ int32_t row_off(uint64_t r) { return (int32_t)(uint32_t)r; }
static __device__ __forceinline__ uint32_t row_deg(uint64_t r) { return (uint32_t)(r >> 32); }

// Bit b of the result is set when byte b of the 16 bytes is not InTree
// (InTree bytes have top bits == epoch | InTree).  Per 4-byte word: SIMD byte
// compare, then bit 7 of each byte gathered into 4 bits by one multiply.
static __device__ __forceinline__ uint32_t gather4(uint32_t eq) { return ((((eq >> 7) & 0x01010101u) * 0x01020408u) >> 24) & 0xFu; }
static __device__ __forceinline__ uint32_t not_tree_mask(ulonglong2 q, uint32_t ep)
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
static __device__ __forceinline__ void pq_set(ulonglong2 &pq, int32_t chunk, uint32_t u, uint32_t b)
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
static __device__ __forceinline__ void commit_one(uint8_t *st, uint32_t e, uint32_t ep, ulonglong2 &pq, int32_t chunk)
{
    const uint32_t b = ep | kBTree | (e >> kEntryShift);
    st[e & kNodeMask] = (uint8_t)b;
    pq_set(pq, chunk, e & kNodeMask, b);
}
static __device__ __forceinline__ void commit_path(uint8_t *st, const uint32_t *stk, uint32_t sp, uint32_t ep,
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
static __device__ __forceinline__ uint32_t erase_loop(uint8_t *st, const uint32_t *stk, uint32_t sp, uint32_t ep, uint32_t h,
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

// The table follows the `cap` stack entries of the slot.
static __device__ __forceinline__ unsigned long long *tbl_of(uint32_t *stk, uint32_t cap)
{
    return reinterpret_cast<unsigned long long *>(stk + cap);
}

// Entry key: node + 1 in bits 0..27 (node < 2^27), the kind of count in bits
// 28..29 (kTblDraws: Wilson draws; kTblUPath / kTblPiPath: departures of the
// uniform-start / pi-start loop-included path).
constexpr uint32_t kTblDraws = 0u, kTblUPath = 1u, kTblPiPath = 2u;
static __device__ __forceinline__ uint32_t tbl_key(uint32_t node, uint32_t kind) { return (node + 1u) | (kind << 28); }

static __device__ __forceinline__ uint32_t tbl_home(uint32_t key, uint32_t log2)
{
    return (key * 2654435761u) >> (32u - log2);
}

// Count of (node, kind) in the current sample (tag); 0 if absent.
static __device__ __forceinline__ uint32_t tbl_get(const unsigned long long *tbl, uint32_t log2, uint32_t node,
                                                   uint32_t kind, uint32_t tag)
{
    const uint32_t mask = (1u << log2) - 1u;
    const uint32_t key = tbl_key(node, kind);
    uint32_t s = tbl_home(key, log2);
    for (uint32_t q = 0; q < kTblProbes; ++q, s = (s + 1u) & mask) {
        const unsigned long long e = tbl[s];
        if (((uint32_t)e >> 24) != tag) break;                 // empty for this sample
        if ((uint32_t)(e >> 32) == key) return (uint32_t)e & 0xFFFFFFu;
    }
    return 0u;
}

// Sets the count of (node, kind), inserting it; false when its probe run is full.
static __device__ __forceinline__ bool tbl_put(unsigned long long *tbl, uint32_t log2, uint32_t node, uint32_t kind,
                                               uint32_t k, uint32_t tag)
{
    const uint32_t mask = (1u << log2) - 1u;
    const uint32_t key = tbl_key(node, kind);
    uint32_t s = tbl_home(key, log2);
    for (uint32_t q = 0; q < kTblProbes; ++q, s = (s + 1u) & mask) {
        const unsigned long long e = tbl[s];
        if (((uint32_t)e >> 24) != tag || (uint32_t)(e >> 32) == key) {
            tbl[s] = ((unsigned long long)key << 32) | ((unsigned long long)tag << 24) | k;
            return true;
        }
    }
    return false;
}

static __device__ __forceinline__ void tbl_clear(unsigned long long *tbl, uint32_t log2)
{
    uint4 *t = reinterpret_cast<uint4 *>(tbl);
    for (uint32_t j = 0; j < (1u << log2) / 2u; ++j) t[j] = make_uint4(0u, 0u, 0u, 0u);
}

// Next sample's tag; clears the table when the tags wrap around.
static __device__ __forceinline__ uint32_t tbl_next_tag(unsigned long long *tbl, uint32_t log2, uint32_t tag)
{
    if (tag >= 255u) {
        tbl_clear(tbl, log2);
        return 1u;
    }
    return tag + 1u;
}

// Withdraws a partly run sample: subtracts the k - 1 repeat visits every
// node of the sample has contributed (and, with the control variate, the
// potentials h1[w] of its k draws, recomputed from their Philox keys) and
// marks all bytes "current epoch, untouched", so that the next sample (next
// epoch) reads them as stale.
static __device__ void withdraw_sample(uint8_t *st, int32_t n, uint32_t ep, unsigned long long *rep1, const int2 *rowinfo,
                                const int32_t *col, const long long *h1, unsigned long long *a1, uint32_t i,
                                uint32_t key0, uint32_t key1, const unsigned long long *tbl, uint32_t log2,
                                uint32_t tag)
{
    for (int32_t base = 0; base < n; base += 16) {
        ulonglong2 q = *reinterpret_cast<ulonglong2 *>(st + base);
#pragma unroll
        for (int b = 0; b < 16; ++b) {
            const uint32_t byte = (uint32_t)(((b < 8 ? q.x : q.y) >> (8 * (b & 7))) & 0xFFu);
            const uint32_t k = b_k(byte, ep);          // kKSat for a node in the table: its first 31 draws
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
    // Draws kKSat .. k-1 of the nodes in the count table (exactly the nodes
    // whose byte held kKSat).
    for (uint32_t j = 0; j < (1u << log2); ++j) {
        const unsigned long long e = tbl[j];
        if (((uint32_t)e >> 24) != tag || (uint32_t)(e >> 60) != kTblDraws) continue;
        const uint32_t node = (uint32_t)(e >> 32) - 1u, k = (uint32_t)e & 0xFFFFFFu;
        if ((int32_t)node >= n || k <= kKSat) continue;
        atomicAdd(&rep1[node], (unsigned long long)(-(long long)(k - kKSat)));
        if (h1) {
            const int2 r = rowinfo[node];
            long long sub = 0;
            for (uint32_t d = kKSat; d < k; ++d) {
                const uint64_t x = lap::philox_r64(node, d, i, 0u, key0, key1);
                sub += h1[col[r.x + (int64_t)lap::below(x, (uint64_t)r.y)]];
            }
            atomicAdd(&a1[node], (unsigned long long)(-sub));
        }
    }
}

// Loop-included paths (paths taken on the sample's own stacks): each node has
// one more byte in a second region of the slot, reset chunk by chunk while
// the Wilson scan passes over it: bits 0..3 count the departures of the
// uniform-start path from the node, bits 4..7 those of the pi-start path; 15
// means "15 or more, see the table" (kinds kTblUPath and kTblPiPath).
constexpr uint32_t kPathSat = 15u;

// Departure count of `nib` (0: uniform path, 1: pi path) of a node.
static __device__ __forceinline__ uint32_t path_count(uint32_t byte, uint32_t nib, const unsigned long long *tbl,
                                                      uint32_t log2, uint32_t node, uint32_t tag)
{
    const uint32_t c = (byte >> (4u * nib)) & 0xFu;
    return c < kPathSat ? c : tbl_get(tbl, log2, node, kTblUPath + nib, tag);
}

// Withdraws what the loop-included paths of a sample added before it was
// withdrawn: every departure of the uniform-start path added one pass to
// cnt2; every departure of the pi-start path added h2[w] to a2 and one to p2
// (control variate).
static __device__ void withdraw_paths(const uint8_t *pr, int32_t n, const unsigned long long *tbl, uint32_t log2,
                                      uint32_t tag, unsigned long long *cnt2, const int2 *rowinfo,
                                      const int32_t *col, const long long *h2, unsigned long long *a2,
                                      unsigned long long *p2, uint32_t i, uint32_t key0, uint32_t key1)
{
    for (int32_t c0 = 0; c0 < n; c0 += 16) {
        const ulonglong2 q = *reinterpret_cast<const ulonglong2 *>(pr + c0);
        if ((q.x | q.y) == 0ull) continue;
        for (int b = 0; b < 16; ++b) {
            const int32_t u = c0 + b;
            if (u >= n) break;
            const uint32_t byte = (uint32_t)(((b < 8 ? q.x : q.y) >> (8 * (b & 7))) & 0xFFu);
            if (!byte) continue;
            const uint32_t ju = path_count(byte, 0u, tbl, log2, (uint32_t)u, tag);
            const uint32_t jp = path_count(byte, 1u, tbl, log2, (uint32_t)u, tag);
            if (ju) atomicAdd(&cnt2[u], (unsigned long long)(-(long long)ju));
            if (jp && h2) {
                const int2 r = rowinfo[u];
                long long sub = 0;
                for (uint32_t d = 0; d < jp; ++d) {
                    const uint64_t x = lap::philox_r64((uint32_t)u, d, i, 0u, key0, key1);
                    sub += h2[col[r.x + (int64_t)lap::below(x, (uint64_t)r.y)]];
                }
                atomicAdd(&a2[u], (unsigned long long)(-sub));
                atomicAdd(&p2[u], (unsigned long long)(-(long long)jp));
            }
        }
    }
}

}  // namespace lap_compact
