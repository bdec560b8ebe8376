// Batched LEWalk sampler: many graphs, each with its own root, in one
// persistent launch.  Every sample of every graph is the same computation as
// in sampler_compact.cu (one Wilson LE_v run, one uniform-start and one
// pi-start v-absorbed walk; Alg. 2 and Alg. 4), with the same Philox keying,
// so graph g's counts equal those of a single-graph run with the same seed
// and sample ids 0 .. count-1.
//
// Work is a queue of units {graph, first sample}, each up to `claim`
// consecutive samples of one graph, in the order the host chose (largest
// graphs first by default).  A lane claims a unit, runs its samples one by
// one in its slot (one state byte per node of the largest graph plus a path
// stack), then claims the next unit, whatever graph it belongs to.
//
// Slots change graphs, so the epoch trick of the single-graph kernel (a byte
// whose epoch bit differs from the lane's reads "untouched") needs one more
// invariant: bytes [0, extent) of the slot carry the lane's current epoch,
// where extent is the node count of the lane's last sample.  Before a sample
// on a graph with n > extent, bytes [extent, n) are stamped with the current
// epoch; then the epoch flips and every byte in [0, n) reads untouched.  A
// fresh slot has extent 0, so the workspace never needs clearing.
//
// Per graph: the count of finished samples, and the globaltimer value when
// its last sample finished (completion time).  Samples the compact state
// cannot represent are withdrawn exactly (see compact_state.cuh) and listed
// as {graph, id} for the host to re-run with the 8-byte kernel.
#include "compact_state.cuh"

namespace {

using namespace lap_compact;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bytes [from, to) of a slot := `ep` (epoch only: not InTree, not on the path, k = 0).
__device__ void stamp(uint8_t *st, int32_t from, int32_t to, uint32_t ep)
{
    const unsigned long long fill = 0x0101010101010101ull * (unsigned long long)ep;
    int32_t a = from;
    for (; a < to && (a & 15); ++a) st[a] = (uint8_t)ep;
    for (; a + 16 <= to; a += 16) *reinterpret_cast<ulonglong2 *>(st + a) = make_ulonglong2(fill, fill);
    for (; a < to; ++a) st[a] = (uint8_t)ep;
}

// PROBE: autotuner launches; each lane stops `window_ns` after it starts
// (possibly inside a sample) and adds the walk steps it took to ctl->steps.
// Counts and slot state are scratch afterwards.
template <bool PROBE, bool PATHS>
__global__ void __launch_bounds__(256, 2) lewalk_batch_kernel(LapBatchLaunch p)
{
    if (threadIdx.x == 0) atomicMin(&p.ctl->t0, global_ns());
    const uint64_t slot = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (slot >= p.lanes) return;
    uint8_t *__restrict__ st = reinterpret_cast<uint8_t *>(p.ws) + slot * p.slot_bytes;
    uint8_t *__restrict__ pr = st + p.n_pad;     // path departure counts (loop-included paths)
    uint32_t *__restrict__ stk = reinterpret_cast<uint32_t *>(st + (PATHS ? 2u : 1u) * p.n_pad);
    const uint32_t cap = p.stack_cap;
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);
    const uint64_t keep = policy_evict_last();
    const unsigned long long t_stop = PROBE ? global_ns() + p.window_ns : 0ull;

    const uint32_t meta = p.slot_meta[slot];
    uint32_t ep = (meta >> 31) ? kBEpoch : 0u;
    int32_t extent = (int32_t)(meta & 0x7FFFFFFFu);

    // The graph of the current unit.
    int32_t gi = -1, n = 0, v = 0;
    const int2 *__restrict__ rowinfo = nullptr;
    const int32_t *__restrict__ col = nullptr;
    unsigned long long *rep1 = nullptr, *cnt2 = nullptr;
    int64_t arcs = 0;
    uint64_t limit = 0;
    uint32_t count_g = 0, unit_end = 0, ustart = 0;

    uint32_t phase = P_CLAIM;
    uint32_t i = 0;
    int32_t s = 0;
    int32_t chunk = -1;
    int32_t h = 0;
    uint32_t sp = 0;
    uint32_t e0 = 0;
    uint32_t pa = 0;
    uint64_t pb = 0;
    ulonglong2 pq = make_ulonglong2(0, 0);
    uint64_t y1 = 0, t = 0, y2 = 0;
    unsigned long long probe_steps = 0;
    uint32_t iter = 0;
    unsigned int bad = 0;
    const uint32_t tlog = p.tbl_log2;
    uint32_t tag = 255u;      // count-table tag of the current sample (the first claim clears the table)

    for (;;) {
        if (PROBE && ((++iter & 255u) == 0u) && global_ns() > t_stop) break;
        if (phase == P_WALK) {
            const int32_t off = row_off(pb);
            const uint32_t deg = row_deg(pb);
            int32_t w = ld_col(col + off + (int64_t)lap::below(lap::philox_r64((uint32_t)h, 0u, i, 0u, key0, key1), deg), keep);
            const uint32_t b = pa;
            if (!b_tree(b, ep)) {
                if (b_path(b, ep)) sp = erase_loop(st, stk, sp, ep, (uint32_t)h, pq, chunk);
                uint32_t kh = b_k(b, ep);
                if (kh == kKSat) {
                    kh = tbl_get(tbl_of(stk, cap), tlog, (uint32_t)h, kTblDraws, tag);
                    if (kh < kKSat) { bad |= LAP_DEV_BAD_INDEX; phase = P_CLAIM; continue; }
                }
                if (kh) w = ld_col(col + off + (int64_t)lap::below(lap::philox_r64((uint32_t)h, kh, i, 0u, key0, key1), deg), keep);
                const uint32_t kn = kh + 1u;
                uint32_t kb = kn;
                bool fits = kn <= kKMax && sp < cap;
                if (fits && kn >= kKSat) {
                    kb = kKSat;
                    fits = tbl_put(tbl_of(stk, cap), tlog, (uint32_t)h, kTblDraws, kn, tag);
                }
                if (!fits) {
                    withdraw_sample(st, n, ep, rep1, rowinfo, col, nullptr, nullptr, i, key0, key1, tbl_of(stk, cap), tlog, tag);
                    const unsigned int ix = atomicAdd(&p.ctl->ovf_count, 1u);
                    if (ix < p.ovf_cap) p.ovf[ix] = make_uint2((uint32_t)gi, i);
                    else bad |= LAP_DEV_K_OVERFLOW;
                    if (atomicAdd(&p.done[gi], 1u) + 1u == count_g) p.t_done[gi] = global_ns();
                    phase = P_CLAIM;
                    continue;
                }
                const uint32_t e = (uint32_t)h | (kb << kEntryShift);
                if (sp == 0) e0 = e;
                st_stack(stk + sp, e, keep);
                ++sp;
                st_state(st + h, ep | kBPath | kb);
                pq_set(pq, chunk, (uint32_t)h, ep | kBPath | kb);
                if (kh) atomicAdd(&rep1[h], 1ull);
                if (PROBE) ++probe_steps;
                if (++y1 > limit) { bad |= LAP_DEV_STEP_LIMIT; phase = P_CLAIM; continue; }
                h = w;
                pa = ld_state(st + w);
                pb = ld_row(rowinfo, w, keep);
                continue;
            }
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
            if (s < n) {
                const int32_t base = s & ~15;
                if (base != chunk) {
                    pq = *reinterpret_cast<const ulonglong2 *>(st + base);
                    chunk = base;
                    if (PATHS) *reinterpret_cast<ulonglong2 *>(pr + base) = make_ulonglong2(0ull, 0ull);
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
                    if (PATHS) *reinterpret_cast<ulonglong2 *>(pr + s) = make_ulonglong2(0ull, 0ull);
                    continue;
                }
            }
            phase = P_USTART_IMMEDIATE;
        }
        if (phase == P_USTART_IMMEDIATE) {
            t = 0;
            h = ustart ? (int32_t)(ustart - 1u)
                         : (int32_t)lap::below(lap::philox_r64(0u, 0u, i, 1u, key0, key1), (uint64_t)n);
            if (h != v) {
                if (!PATHS) atomicAdd(&cnt2[h], 1ull);
                pb = ld_row(rowinfo, h, keep);
                phase = P_UWALK;
                continue;
            }
            phase = P_PISTART_IMMEDIATE;
        }
        if (phase == P_UWALK) {
            ++t;
            if (PROBE) ++probe_steps;
            int32_t w;
            if (PATHS) {
                // Loop-included path: departure j from h takes h's stack entry j.
                const uint32_t pbyte = pr[h];
                const uint32_t j = path_count(pbyte, 0u, tbl_of(stk, cap), tlog, (uint32_t)h, tag);
                w = ld_col(col + row_off(pb) + (int64_t)lap::below(lap::philox_r64((uint32_t)h, j, i, 0u, key0, key1), row_deg(pb)), keep);
                const uint32_t jn = j + 1u;
                const uint32_t cn = jn < kPathSat ? jn : kPathSat;
                if (jn >= kPathSat && !tbl_put(tbl_of(stk, cap), tlog, (uint32_t)h, kTblUPath, jn, tag)) {
                    withdraw_sample(st, n, ep, rep1, rowinfo, col, nullptr, nullptr, i, key0, key1, tbl_of(stk, cap), tlog, tag);
                    withdraw_paths(pr, n, tbl_of(stk, cap), tlog, tag, cnt2, rowinfo, col, nullptr, nullptr, nullptr, i, key0, key1);
                    const unsigned int ix = atomicAdd(&p.ctl->ovf_count, 1u);
                    if (ix < p.ovf_cap) p.ovf[ix] = make_uint2((uint32_t)gi, i);
                    else bad |= LAP_DEV_K_OVERFLOW;
                    if (atomicAdd(&p.done[gi], 1u) + 1u == count_g) p.t_done[gi] = global_ns();
                    phase = P_CLAIM;
                    continue;
                }
                // Written after the table accepted a count of 15 or more, so that a
                // withdrawn path finds its departures so far.
                pr[h] = (uint8_t)((pbyte & (0xF0u >> (4u * 0u))) | (cn << (4u * 0u)));
                atomicAdd(&cnt2[h], 1ull);
            } else {
                const uint64_t r = lap::philox_r64((uint32_t)t, 0u, i, 1u, key0, key1);
                w = ld_col(col + row_off(pb) + (int64_t)lap::below(r, row_deg(pb)), keep);
            }
            h = w;
            if (t > limit) { bad |= LAP_DEV_STEP_LIMIT; phase = P_CLAIM; continue; }
            if (h != v) {
                if (!PATHS) atomicAdd(&cnt2[h], 1ull);
                pb = ld_row(rowinfo, h, keep);
                continue;
            }
            phase = P_PISTART_IMMEDIATE;
        }
        if (phase == P_PISTART_IMMEDIATE) {
            y2 = 0;
            h = ld_col(col + (int64_t)lap::below(lap::philox_r64(0u, 0u, i, 2u, key0, key1), (uint64_t)arcs), keep);
            if (h != v) { pb = ld_row(rowinfo, h, keep); phase = P_PIWALK; continue; }
            phase = P_FINISH_IMMEDIATE;
        }
        if (phase == P_PIWALK) {
            ++y2;
            if (PROBE) ++probe_steps;
            if (PATHS) {
                const uint32_t pbyte = pr[h];
                const uint32_t j = path_count(pbyte, 1u, tbl_of(stk, cap), tlog, (uint32_t)h, tag);
                const int32_t w = ld_col(col + row_off(pb) + (int64_t)lap::below(lap::philox_r64((uint32_t)h, j, i, 0u, key0, key1), row_deg(pb)), keep);
                const uint32_t jn = j + 1u;
                const uint32_t cn = jn < kPathSat ? jn : kPathSat;
                if (jn >= kPathSat && !tbl_put(tbl_of(stk, cap), tlog, (uint32_t)h, kTblPiPath, jn, tag)) {
                    withdraw_sample(st, n, ep, rep1, rowinfo, col, nullptr, nullptr, i, key0, key1, tbl_of(stk, cap), tlog, tag);
                    withdraw_paths(pr, n, tbl_of(stk, cap), tlog, tag, cnt2, rowinfo, col, nullptr, nullptr, nullptr, i, key0, key1);
                    const unsigned int ix = atomicAdd(&p.ctl->ovf_count, 1u);
                    if (ix < p.ovf_cap) p.ovf[ix] = make_uint2((uint32_t)gi, i);
                    else bad |= LAP_DEV_K_OVERFLOW;
                    if (atomicAdd(&p.done[gi], 1u) + 1u == count_g) p.t_done[gi] = global_ns();
                    phase = P_CLAIM;
                    continue;
                }
                // Written after the table accepted a count of 15 or more, so that a
                // withdrawn path finds its departures so far.
                pr[h] = (uint8_t)((pbyte & (0xF0u >> (4u * 1u))) | (cn << (4u * 1u)));
                h = w;
            } else {
                const uint64_t r = lap::philox_r64((uint32_t)y2, 0u, i, 2u, key0, key1);
                h = ld_col(col + row_off(pb) + (int64_t)lap::below(r, row_deg(pb)), keep);
            }
            if (y2 > limit) { bad |= LAP_DEV_STEP_LIMIT; phase = P_CLAIM; continue; }
            if (h != v) { pb = ld_row(rowinfo, h, keep); continue; }
            phase = P_FINISH_IMMEDIATE;
        }
        if (phase == P_FINISH_IMMEDIATE) {
            atomicAdd(&p.acc[gi].sum_y1, (unsigned long long)y1);
            atomicAdd(&p.acc[gi].sum_y2, (unsigned long long)y2);
            if (atomicAdd(&p.done[gi], 1u) + 1u == count_g) p.t_done[gi] = global_ns();
            phase = P_CLAIM;
        }
        if (phase == P_CLAIM) {
            if (bad) break;
            if (i + 1u < unit_end) {
                ++i;
            } else {
                const unsigned int q = atomicAdd(&p.ctl->claim, 1u);
                if (q >= p.n_units) break;
                const uint2 u = p.units[q];
                if ((int32_t)u.x != gi) {
                    const LapBatchGraph *d = p.graphs + u.x;
                    gi = (int32_t)u.x;
                    n = d->n;
                    v = d->root;
                    rowinfo = d->rowinfo;
                    col = d->col;
                    rep1 = d->rep1;
                    cnt2 = d->cnt2;
                    arcs = d->arcs;
                    limit = d->step_limit;
                    count_g = d->count;
                    ustart = d->ustart;
                }
                i = u.y;
                unit_end = u.y + p.claim < count_g ? u.y + p.claim : count_g;
            }
            // Bytes [0, n) must carry the current epoch before it flips.
            if (n > extent) stamp(st, extent, n, ep);
            extent = n;
            tag = tbl_next_tag(tbl_of(stk, cap), tlog, tag);
            ep ^= kBEpoch;
            st[v] = (uint8_t)(ep | kBTree);
            s = 0;
            sp = 0;
            y1 = 0;
            chunk = -1;
            phase = P_SCAN;
        }
    }
    if (PROBE) {
        atomicAdd(&p.ctl->steps, probe_steps);
    } else {
        p.slot_meta[slot] = (ep ? 0x80000000u : 0u) | (uint32_t)extent;
    }
    if (bad) atomicOr(&p.ctl->status, bad);
}

}  // namespace

int lap_batch_block(const LapBatchLaunch &p) { return p.block > 0 ? p.block : lap_pick_block(p.lanes, p.num_sms); }

uint64_t lap_batch_resident_lanes(int block, int num_sms)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lewalk_batch_kernel<false, true>, block, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (uint64_t)per_sm * (uint64_t)block * (uint64_t)(num_sms > 0 ? num_sms : 1);
}

cudaError_t lap_launch_batch(const LapBatchLaunch &p, bool probe, cudaStream_t st)
{
    if (p.lanes == 0 || p.n_units == 0) return cudaSuccess;
    const int block = lap_batch_block(p);
    const uint64_t grid = (p.lanes + block - 1) / block;
    if (probe && p.paths) lewalk_batch_kernel<true, true><<<(unsigned)grid, block, 0, st>>>(p);
    else if (probe) lewalk_batch_kernel<true, false><<<(unsigned)grid, block, 0, st>>>(p);
    else if (p.paths) lewalk_batch_kernel<false, true><<<(unsigned)grid, block, 0, st>>>(p);
    else lewalk_batch_kernel<false, false><<<(unsigned)grid, block, 0, st>>>(p);
    return cudaGetLastError();
}
