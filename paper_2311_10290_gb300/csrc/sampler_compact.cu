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
// InTree; counts above 30 go to the lane's count table, see
// compact_state.cuh), and the repeat-visit counter has received exactly
// k - 1 for every node touched so far.  A sample that cannot be represented
// (the count table full, or a loop-erased path longer than the stack) is
// therefore withdrawn exactly: the lane subtracts k - 1 for every node of
// the sample, re-stamps its state bytes with the current epoch (so the next
// sample sees them all as stale), appends the sample id to an overflow list
// and goes on with the next sample.  The host re-runs the listed ids with
// the 8-byte kernel.  Nothing else of a sample is counted before its Wilson
// run completes.
#include "compact_state.cuh"

namespace {

using namespace lap_compact;

// CV: control-variate sums; PATHS: the absorbed walks are loop-included
// paths (LapSampleLaunch::paths).  Separate instantiations keep the plain
// kernel free of the other modes' code.
template <bool CV, bool PATHS>
__global__ void __launch_bounds__(256, CV ? 2 : 4) lewalk_compact_kernel(LapSampleLaunch p)
{
    const uint64_t slot = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (slot >= p.slots) return;
    const int32_t n = p.g.n;
    const int32_t v = p.root;
    const int2 *__restrict__ rowinfo = p.g.rowinfo;
    const int32_t *__restrict__ col = p.g.col;
    uint8_t *__restrict__ st = reinterpret_cast<uint8_t *>(p.ws) + slot * p.slot_bytes;
    uint8_t *__restrict__ pr = st + p.n_pad;     // path departure counts (loop-included paths)
    uint32_t *__restrict__ stk = reinterpret_cast<uint32_t *>(st + (PATHS ? 2u : 1u) * p.n_pad);
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
    const uint32_t tlog = p.tbl_log2;
    uint32_t tag = 255u;      // count-table tag of the current sample (the first claim clears the table)

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
                    withdraw_sample(st, n, ep, p.rep1, rowinfo, col, CV ? p.cv_h1 : nullptr, p.cv_a1, i, key0, key1, tbl_of(stk, cap), tlog, tag);
                    const unsigned int ix = atomicAdd(&p.acc->ovf_count, 1u);
                    if (ix < p.count) p.ovf_ids[ix] = i;
                    phase = P_CLAIM;
                    continue;
                }
                const uint32_t e = (uint32_t)h | (kb << kEntryShift);
                if (sp == 0) e0 = e;
                st_stack(stk + sp, e, keep);
                ++sp;
                st_state(st + h, ep | kBPath | kb);
                pq_set(pq, chunk, (uint32_t)h, ep | kBPath | kb);
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
            // Alg. 2: uniformly sample s in V (or take the fixed start of a
            // single-source row); walk until v, counting passes.
            t = 0;
            h = p.ustart ? (int32_t)(p.ustart - 1u)
                         : (int32_t)lap::below(lap::philox_r64(0u, 0u, i, 1u, key0, key1), (uint64_t)n);
            if (h != v) {
                if (!PATHS) atomicAdd(&p.cnt2[h], 1ull);
                pb = ld_row(rowinfo, h, keep);
                phase = P_UWALK;
                continue;
            }
            phase = P_PISTART_IMMEDIATE;
        }
        if (phase == P_UWALK) {
            ++t;
            int32_t w;
            if (PATHS) {
                // Loop-included path: departure j from h takes h's stack entry j.
                const uint32_t pbyte = pr[h];
                const uint32_t j = path_count(pbyte, 0u, tbl_of(stk, cap), tlog, (uint32_t)h, tag);
                w = ld_col(col + row_off(pb) + (int64_t)lap::below(lap::philox_r64((uint32_t)h, j, i, 0u, key0, key1), row_deg(pb)), keep);
                const uint32_t jn = j + 1u;
                const uint32_t cn = jn < kPathSat ? jn : kPathSat;
                if (jn >= kPathSat && !tbl_put(tbl_of(stk, cap), tlog, (uint32_t)h, kTblUPath, jn, tag)) {
                    withdraw_sample(st, n, ep, p.rep1, rowinfo, col, CV ? p.cv_h1 : nullptr, p.cv_a1, i, key0, key1, tbl_of(stk, cap), tlog, tag);
                    withdraw_paths(pr, n, tbl_of(stk, cap), tlog, tag, p.cnt2, rowinfo, col, CV ? p.cv_h2 : nullptr, p.cv_a2, p.cv_p2, i, key0, key1);
                    const unsigned int ix = atomicAdd(&p.acc->ovf_count, 1u);
                    if (ix < p.count) p.ovf_ids[ix] = i;
                    phase = P_CLAIM;
                    continue;
                }
                // Written after the table accepted a count of 15 or more, so that a
                // withdrawn path finds its departures so far.
                pr[h] = (uint8_t)((pbyte & (0xF0u >> (4u * 0u))) | (cn << (4u * 0u)));
                atomicAdd(&p.cnt2[h], 1ull);
            } else {
                const uint64_t r = lap::philox_r64((uint32_t)t, 0u, i, 1u, key0, key1);
                w = ld_col(col + row_off(pb) + (int64_t)lap::below(r, row_deg(pb)), keep);
            }
            h = w;
            if (t > limit) { bad |= LAP_DEV_STEP_LIMIT; phase = P_CLAIM; continue; }
            if (h != v) {
                if (!PATHS) atomicAdd(&p.cnt2[h], 1ull);
                pb = ld_row(rowinfo, h, keep);
                continue;
            }
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
            int32_t w;
            if (PATHS) {
                const uint32_t pbyte = pr[h];
                const uint32_t j = path_count(pbyte, 1u, tbl_of(stk, cap), tlog, (uint32_t)h, tag);
                w = ld_col(col + row_off(pb) + (int64_t)lap::below(lap::philox_r64((uint32_t)h, j, i, 0u, key0, key1), row_deg(pb)), keep);
                const uint32_t jn = j + 1u;
                const uint32_t cn = jn < kPathSat ? jn : kPathSat;
                if (jn >= kPathSat && !tbl_put(tbl_of(stk, cap), tlog, (uint32_t)h, kTblPiPath, jn, tag)) {
                    withdraw_sample(st, n, ep, p.rep1, rowinfo, col, CV ? p.cv_h1 : nullptr, p.cv_a1, i, key0, key1, tbl_of(stk, cap), tlog, tag);
                    withdraw_paths(pr, n, tbl_of(stk, cap), tlog, tag, p.cnt2, rowinfo, col, CV ? p.cv_h2 : nullptr, p.cv_a2, p.cv_p2, i, key0, key1);
                    const unsigned int ix = atomicAdd(&p.acc->ovf_count, 1u);
                    if (ix < p.count) p.ovf_ids[ix] = i;
                    phase = P_CLAIM;
                    continue;
                }
                // Written after the table accepted a count of 15 or more, so that a
                // withdrawn path finds its departures so far.
                pr[h] = (uint8_t)((pbyte & (0xF0u >> (4u * 1u))) | (cn << (4u * 1u)));
            } else {
                const uint64_t r = lap::philox_r64((uint32_t)y2, 0u, i, 2u, key0, key1);
                w = ld_col(col + row_off(pb) + (int64_t)lap::below(r, row_deg(pb)), keep);
            }
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
    const bool cv = p.cv_h1 || p.cv_h2;
    if (cv && p.paths) lewalk_compact_kernel<true, true><<<(unsigned)grid, block, 0, st>>>(p);
    else if (cv) lewalk_compact_kernel<true, false><<<(unsigned)grid, block, 0, st>>>(p);
    else if (p.paths) lewalk_compact_kernel<false, true><<<(unsigned)grid, block, 0, st>>>(p);
    else lewalk_compact_kernel<false, false><<<(unsigned)grid, block, 0, st>>>(p);
    return cudaGetLastError();
}
