// Host side of include/lap_batch.h: packed arenas of many graphs, the work
// queue, CUDA-graph capture of one run (resets, persistent sampler, finalize),
// re-runs of withdrawn samples, and the autotuner.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "lap_batch.h"
#include "lap_internal.h"

struct lap_batch {
    int device = 0;
    int num_sms = 0;
    int32_t G = 0;
    std::vector<int32_t> n, roots;
    std::vector<int64_t> arcs, node_off, arc_off;   // per-graph offsets of counts and outputs
    std::vector<int32_t> src;                        // graph whose CSR arena region graph g shares (itself if first)
    std::vector<int64_t> csr_node_off, csr_arc_off;  // graph g's row records and columns in the CSR arenas
    int64_t csr_nodes = 0, csr_arcs = 0;
    int64_t total_n = 0, total_arcs = 0;
    int32_t max_n = 0;

    int32_t *d_col = nullptr;
    int2 *d_rowinfo = nullptr;
    unsigned long long *d_rep1 = nullptr, *d_cnt2 = nullptr, *d_scratch = nullptr;
    double *d_ldiag = nullptr, *d_ecc = nullptr, *d_red = nullptr;
    LapBatchGraph *d_graphs = nullptr;
    std::vector<LapBatchGraph> h_graphs;
    LapDevAcc *d_acc = nullptr;
    unsigned int *d_done = nullptr;
    unsigned long long *d_tdone = nullptr;
    LapBatchCtl *d_ctl = nullptr;
    uint2 *d_units = nullptr;
    uint64_t units_cap = 0;
    uint32_t n_units = 0;
    uint2 *d_ovf = nullptr;
    unsigned int *d_rerun_ids = nullptr;
    uint32_t ovf_cap = 0;
    unsigned int *d_slot_meta = nullptr;
    uint64_t meta_cap = 0;
    bool meta_dirty = true;              // slot extents must restart from 0 before the next run

    void *ws = nullptr;
    uint64_t ws_bytes = 0;
    bool ws_owned = false;

    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t rerun_streams[8] = {};
    cudaEvent_t rerun_done[8] = {};
    cudaGraphExec_t exec = nullptr;
    bool key_valid = false;
    uint64_t key_samples = 0, key_seed = 0, key_lanes = 0;
    uint32_t key_claim = 0, key_stack = 0, key_paths = 0;
    int key_order = -1, key_block = -1;
    int64_t captures = 0;

    uint64_t lanes_opt = 0;
    uint32_t claim_opt = 1;
    int order_opt = 0;
    int block_opt = 0;
    uint32_t stack_opt = 0;
    uint32_t paths_opt = 0;

    uint64_t omega = 0;
    uint64_t seed = 0;
    bool ran = false;
    bool checked = false;
    int64_t reruns = 0;

    lap_status sticky = LAP_OK;
    std::string err = "no error";
};

namespace {

thread_local std::string g_batch_error = "no error";
constexpr int kRerunStreams = 8;

lap_status bfail(lap_batch *b, lap_status s, const std::string &msg)
{
    if (b) b->err = msg;
    else g_batch_error = msg;
    return s;
}

lap_status bcuda(lap_batch *b, cudaError_t e, const char *where)
{
    if (b) b->sticky = LAP_ERR_CUDA;
    return bfail(b, LAP_ERR_CUDA, std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e));
}

#define B_CUDA(b, call)                                          \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return bcuda((b), e_, #call);     \
    } while (0)

template <class T>
cudaError_t balloc(T **p, size_t count)
{
    return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (count > 0 ? count : 1));
}

void free_batch(lap_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (int k = 0; k < 8; ++k) {
        if (b->rerun_streams[k]) cudaStreamDestroy(b->rerun_streams[k]);
        if (b->rerun_done[k]) cudaEventDestroy(b->rerun_done[k]);
    }
    cudaFree(b->d_col);
    cudaFree(b->d_rowinfo);
    cudaFree(b->d_rep1);
    cudaFree(b->d_cnt2);
    cudaFree(b->d_scratch);
    cudaFree(b->d_ldiag);
    cudaFree(b->d_ecc);
    cudaFree(b->d_red);
    cudaFree(b->d_graphs);
    cudaFree(b->d_acc);
    cudaFree(b->d_done);
    cudaFree(b->d_tdone);
    cudaFree(b->d_ctl);
    cudaFree(b->d_units);
    cudaFree(b->d_ovf);
    cudaFree(b->d_rerun_ids);
    cudaFree(b->d_slot_meta);
    if (b->ws_owned) cudaFree(b->ws);
}

uint64_t step_limit_of(int32_t n) { return (1ull << 20) + 1024ull * (uint64_t)n; }

uint32_t stack_cap_of(const lap_batch *b)
{
    if (b->stack_opt) return b->stack_opt;
    uint64_t c = 1024;
    while (c * c < 256ull * (uint64_t)b->max_n && c < (1u << 20)) c <<= 1;
    return (uint32_t)c;
}

uint64_t n_pad_of(const lap_batch *b) { return ((uint64_t)b->max_n + 255ull) & ~255ull; }

uint64_t slot_bytes_of(const lap_batch *b)
{
    return ((b->paths_opt ? 2ull : 1ull) * n_pad_of(b) + 4ull * stack_cap_of(b) + (8ull << lap_table_log2(b->max_n)) +
            255ull) & ~255ull;
}

// Work units in claim order (shared by lap_batch_run and lap_batch_schedule).
void build_units(int32_t G, const int32_t *n, int order, uint64_t samples, uint32_t claim, std::vector<uint2> &out)
{
    std::vector<int32_t> gorder((size_t)G);
    std::iota(gorder.begin(), gorder.end(), 0);
    if (order == 0)
        std::stable_sort(gorder.begin(), gorder.end(), [&](int32_t a, int32_t c) { return n[a] > n[c]; });
    else if (order == 1)
        std::stable_sort(gorder.begin(), gorder.end(), [&](int32_t a, int32_t c) { return n[a] < n[c]; });
    out.clear();
    for (int32_t g : gorder)
        for (uint64_t f = 0; f < samples; f += claim) out.push_back(make_uint2((uint32_t)g, (uint32_t)f));
}

lap_status check_handle(lap_batch *b)
{
    if (!b) return bfail(nullptr, LAP_ERR_INVALID_ARG, "NULL handle");
    return b->sticky;
}

// Lanes for the next run: the workspace's slots, the resident-thread
// capacity of the sampler, the lane option and the number of samples.
uint64_t lanes_for(const lap_batch *b, uint64_t samples, uint64_t lanes_opt, int *block_out)
{
    uint64_t lanes = b->ws ? b->ws_bytes / slot_bytes_of(b) : 0;
    if (lanes > b->meta_cap) lanes = b->meta_cap;
    if (lanes_opt && lanes_opt < lanes) lanes = lanes_opt;
    const uint64_t total = samples * (uint64_t)b->G;
    if (total && lanes > total) lanes = total;
    int block = b->block_opt > 0 ? b->block_opt : lap_pick_block(lanes, b->num_sms);
    const uint64_t resident = lap_batch_resident_lanes(block, b->num_sms);
    if (resident && lanes > resident) {
        lanes = resident;
        block = b->block_opt > 0 ? b->block_opt : lap_pick_block(lanes, b->num_sms);
    }
    if (block_out) *block_out = block;
    return lanes;
}

lap_status ensure_workspace(lap_batch *b)
{
    const uint64_t per = slot_bytes_of(b);
    if (!b->ws) {
        size_t free_b = 0, total_b = 0;
        B_CUDA(b, cudaMemGetInfo(&free_b, &total_b));
        uint64_t want = (uint64_t)free_b / 2;
        const uint64_t cap = per * lap_batch_resident_lanes(32, b->num_sms);
        if (cap && want > cap) want = cap;
        want &= ~255ull;
        if (want < per) return bfail(b, LAP_ERR_OOM, "not enough device memory for one lane's Wilson state");
        cudaError_t e = cudaMalloc(&b->ws, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b->ws = nullptr;
            return bfail(b, LAP_ERR_OOM, "workspace allocation failed");
        }
        b->ws_bytes = want;
        b->ws_owned = true;
        b->meta_dirty = true;
    }
    const uint64_t slots = b->ws_bytes / per;
    if (slots == 0) return bfail(b, LAP_ERR_OOM, "workspace smaller than one lane's Wilson state");
    if (slots > b->meta_cap) {
        cudaFree(b->d_slot_meta);
        b->d_slot_meta = nullptr;
        b->meta_cap = 0;
        if (balloc(&b->d_slot_meta, slots) != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, LAP_ERR_OOM, "slot table allocation failed");
        }
        b->meta_cap = slots;
        b->meta_dirty = true;
    }
    if (b->meta_dirty) {
        B_CUDA(b, cudaMemsetAsync(b->d_slot_meta, 0, sizeof(unsigned int) * b->meta_cap, b->stream));
        b->meta_dirty = false;
    }
    return LAP_OK;
}

// Descriptors with this run's sample count, and the unit queue.
lap_status upload_plan(lap_batch *b, uint64_t samples, uint32_t claim)
{
    for (auto &d : b->h_graphs) d.count = (uint32_t)samples;
    B_CUDA(b, cudaMemcpyAsync(b->d_graphs, b->h_graphs.data(), sizeof(LapBatchGraph) * b->h_graphs.size(),
                              cudaMemcpyHostToDevice, b->stream));
    std::vector<uint2> units;
    build_units(b->G, b->n.data(), b->order_opt, samples, claim, units);
    if (units.size() > b->units_cap) {
        cudaFree(b->d_units);
        b->d_units = nullptr;
        b->units_cap = 0;
        if (balloc(&b->d_units, units.size()) != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, LAP_ERR_OOM, "work-unit queue allocation failed");
        }
        b->units_cap = units.size();
    }
    B_CUDA(b, cudaMemcpyAsync(b->d_units, units.data(), sizeof(uint2) * units.size(), cudaMemcpyHostToDevice, b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));      // the host vectors go out of scope
    b->n_units = (uint32_t)units.size();
    return LAP_OK;
}

LapBatchLaunch make_launch(const lap_batch *b, uint64_t seed, uint64_t lanes, uint32_t claim, int block)
{
    LapBatchLaunch p;
    memset(&p, 0, sizeof(p));
    p.graphs = b->d_graphs;
    p.units = b->d_units;
    p.n_units = b->n_units;
    p.claim = claim;
    p.seed = seed;
    p.lanes = lanes;
    p.ws = b->ws;
    p.slot_bytes = slot_bytes_of(b);
    p.n_pad = n_pad_of(b);
    p.tbl_log2 = lap_table_log2(b->max_n);
    p.stack_cap = (uint32_t)((p.slot_bytes - (b->paths_opt ? 2ull : 1ull) * p.n_pad - (8ull << p.tbl_log2)) / 4ull);
    p.slot_meta = b->d_slot_meta;
    p.acc = b->d_acc;
    p.done = b->d_done;
    p.t_done = b->d_tdone;
    p.ctl = b->d_ctl;
    p.ovf = b->d_ovf;
    p.ovf_cap = b->ovf_cap;
    p.block = block;
    p.num_sms = b->num_sms;
    p.paths = b->paths_opt;
    return p;
}

// Captures one run: counter resets, the sampler, the finalize of every graph.
lap_status capture(lap_batch *b, uint64_t samples, uint64_t seed, uint64_t lanes, uint32_t claim, int block)
{
    if (b->exec) {
        B_CUDA(b, cudaStreamSynchronize(b->stream));
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    b->key_valid = false;
    lap_status s = upload_plan(b, samples, claim);
    if (s != LAP_OK) return s;
    const LapBatchLaunch p = make_launch(b, seed, lanes, claim, block);
    cudaStream_t cs = b->cap_stream;
    B_CUDA(b, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const size_t nb = sizeof(unsigned long long) * (size_t)b->total_n;
    cudaError_t e = cudaMemsetAsync(b->d_rep1, 0, nb, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_cnt2, 0, nb, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_acc, 0, sizeof(LapDevAcc) * (size_t)b->G, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_done, 0, sizeof(unsigned int) * (size_t)b->G, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_tdone, 0, sizeof(unsigned long long) * (size_t)b->G, cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ctl, 0, sizeof(LapBatchCtl), cs);
    if (e == cudaSuccess) e = cudaMemsetAsync(&b->d_ctl->t0, 0xFF, sizeof(unsigned long long), cs);
    if (e == cudaSuccess) e = lap_launch_batch(p, false, cs);
    if (e == cudaSuccess) e = lap_launch_finalize_batch(b->d_graphs, b->G, b->max_n, samples, b->d_red, cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        b->exec = nullptr;
        return bcuda(b, e, "capturing the batch run");
    }
    b->key_valid = true;
    b->key_samples = samples;
    b->key_seed = seed;
    b->key_lanes = lanes;
    b->key_claim = claim;
    b->key_order = b->order_opt;
    b->key_block = block;
    b->key_stack = stack_cap_of(b);
    b->key_paths = b->paths_opt;
    ++b->captures;
    return LAP_OK;
}

// Re-runs withdrawn samples with the 8-byte kernel, graph by graph, then
// finalizes every graph again.
lap_status rerun_withdrawn(lap_batch *b, uint32_t count)
{
    if (count > b->ovf_cap) return bfail(b, LAP_ERR_CUDA, "internal error: overflow list exceeded");
    std::vector<uint2> ovf(count);
    B_CUDA(b, cudaMemcpyAsync(ovf.data(), b->d_ovf, sizeof(uint2) * count, cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    std::stable_sort(ovf.begin(), ovf.end(), [](const uint2 &a, const uint2 &c) { return a.x < c.x; });
    std::vector<unsigned int> ids(count);
    for (uint32_t k = 0; k < count; ++k) ids[k] = ovf[k].y;
    B_CUDA(b, cudaMemcpyAsync(b->d_rerun_ids, ids.data(), sizeof(unsigned int) * count, cudaMemcpyHostToDevice, b->stream));
    // Graphs with withdrawn samples are packed into the workspace side by
    // side (one lane per sample where it fits) and re-run concurrently on a
    // few streams; groups that do not fit together run one after another.
    struct Job { uint32_t g, a, c; uint64_t slots, ws_off, meta_off; };
    std::vector<Job> group;
    uint64_t ws_used = 0, meta_used = 0;
    cudaEvent_t ready = nullptr;
    B_CUDA(b, cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    auto flush = [&]() -> lap_status {
        if (group.empty()) return LAP_OK;
        B_CUDA(b, cudaEventRecord(ready, b->stream));
        for (size_t j = 0; j < group.size(); ++j) {
            const Job &jb = group[j];
            cudaStream_t st = b->rerun_streams[j % kRerunStreams];
            B_CUDA(b, cudaStreamWaitEvent(st, ready, 0));
            const LapBatchGraph &d = b->h_graphs[jb.g];
            char *ws = reinterpret_cast<char *>(b->ws) + jb.ws_off;
            B_CUDA(b, cudaMemsetAsync(ws, 0, jb.slots * 8ull * (uint64_t)d.n, st));
            B_CUDA(b, cudaMemsetAsync(b->d_slot_meta + jb.meta_off, 0, sizeof(unsigned int) * jb.slots, st));
            B_CUDA(b, cudaMemsetAsync(&b->d_acc[jb.g].claim, 0, sizeof(unsigned int), st));
            LapSampleLaunch p;
            memset(&p, 0, sizeof(p));
            p.g = LapDevGraph{d.rowinfo, d.col, d.n, d.arcs};
            p.root = d.root;
            p.seed = b->seed;
            p.first = 0;
            p.count = jb.c;
            p.slots = jb.slots;
            p.ws = ws;
            p.slot_epoch = b->d_slot_meta + jb.meta_off;
            p.rep1 = d.rep1;
            p.cnt2 = d.cnt2;
            p.acc = b->d_acc + jb.g;
            p.step_limit = d.step_limit;
            p.num_sms = b->num_sms;
            p.ids = b->d_rerun_ids + jb.a;
            p.paths = b->paths_opt;
            p.ustart = d.ustart;
            B_CUDA(b, lap_launch_sample(p, st));
        }
        for (int k = 0; k < kRerunStreams && k < (int)group.size(); ++k) {
            B_CUDA(b, cudaEventRecord(b->rerun_done[k], b->rerun_streams[k]));
            B_CUDA(b, cudaStreamWaitEvent(b->stream, b->rerun_done[k], 0));
        }
        group.clear();
        ws_used = meta_used = 0;
        return LAP_OK;
    };
    if (!b->rerun_streams[0]) {
        for (int k = 0; k < kRerunStreams; ++k) {
            B_CUDA(b, cudaStreamCreateWithFlags(&b->rerun_streams[k], cudaStreamNonBlocking));
            B_CUDA(b, cudaEventCreateWithFlags(&b->rerun_done[k], cudaEventDisableTiming));
        }
    }
    lap_status fs = LAP_OK;
    for (uint32_t a = 0; a < count && fs == LAP_OK;) {
        uint32_t c = a;
        const uint32_t g = ovf[a].x;
        while (c < count && ovf[c].x == g) ++c;
        if (g >= (uint32_t)b->G) { fs = bfail(b, LAP_ERR_CUDA, "internal error: overflow entry names no graph"); break; }
        const uint64_t per = 8ull * (uint64_t)b->n[g];
        uint64_t slots = c - a;
        if (slots * per > b->ws_bytes) slots = b->ws_bytes / per;
        if (slots > b->meta_cap) slots = b->meta_cap;
        if (slots == 0) { fs = bfail(b, LAP_ERR_OOM, "workspace too small to re-run a withdrawn sample"); break; }
        const uint64_t bytes = (slots * per + 255ull) & ~255ull;
        if (ws_used + bytes > b->ws_bytes || meta_used + slots > b->meta_cap) fs = flush();
        if (fs != LAP_OK) break;
        group.push_back(Job{g, a, c - a, slots, ws_used, meta_used});
        ws_used += bytes;
        meta_used += slots;
        a = c;
    }
    if (fs == LAP_OK) fs = flush();
    cudaEventDestroy(ready);
    if (fs != LAP_OK) return fs;
    b->meta_dirty = true;                    // the slots now hold 8-byte states
    B_CUDA(b, cudaMemsetAsync(b->d_slot_meta, 0, sizeof(unsigned int) * b->meta_cap, b->stream));
    b->meta_dirty = false;
    B_CUDA(b, lap_launch_finalize_batch(b->d_graphs, b->G, b->max_n, b->omega, b->d_red, b->stream));
    std::vector<LapDevAcc> acc((size_t)b->G);
    B_CUDA(b, cudaMemcpyAsync(acc.data(), b->d_acc, sizeof(LapDevAcc) * acc.size(), cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    for (int32_t g = 0; g < b->G; ++g)
        if (acc[(size_t)g].status & LAP_DEV_STEP_LIMIT) {
            b->sticky = LAP_ERR_STEP_LIMIT;
            return bfail(b, LAP_ERR_STEP_LIMIT, "graph " + std::to_string(g) + ": a re-run sample exceeded the step budget");
        }
    b->reruns = count;
    return LAP_OK;
}

// Synchronises after a run; turns device status into errors; re-runs
// withdrawn samples (once per run).
lap_status finish(lap_batch *b)
{
    lap_status s = check_handle(b);
    if (s != LAP_OK) return s;
    if (!b->ran) return bfail(b, LAP_ERR_NO_SAMPLES, "lap_batch_run has not been called");
    if (b->checked) return LAP_OK;
    LapBatchCtl c;
    B_CUDA(b, cudaMemcpyAsync(&c, b->d_ctl, sizeof(c), cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    if (c.status & LAP_DEV_STEP_LIMIT) {
        b->sticky = LAP_ERR_STEP_LIMIT;
        b->meta_dirty = true;
        return bfail(b, LAP_ERR_STEP_LIMIT, "a sample exceeded its graph's step budget (2^20 + 1024 n)");
    }
    if (c.status) {
        b->sticky = LAP_ERR_CUDA;
        b->meta_dirty = true;
        return bfail(b, LAP_ERR_CUDA, "internal error: sampler status " + std::to_string(c.status));
    }
    b->reruns = 0;
    if (c.ovf_count) {
        s = rerun_withdrawn(b, c.ovf_count);
        if (s != LAP_OK) return s;
    }
    b->checked = true;
    return LAP_OK;
}

}  // namespace

extern "C" {

const char *lap_batch_last_error(const lap_batch *b) { return b ? b->err.c_str() : g_batch_error.c_str(); }

lap_status lap_batch_schedule(int32_t n_graphs, const int32_t *n, int32_t order, uint64_t samples, uint32_t claim,
                              uint32_t *unit_graph, uint32_t *unit_first, uint64_t cap, uint64_t *n_units)
{
    if (n_graphs < 1 || !n || !n_units || claim == 0 || order < 0 || order > 2 || samples == 0)
        return bfail(nullptr, LAP_ERR_INVALID_ARG, "bad schedule arguments");
    std::vector<uint2> units;
    build_units(n_graphs, n, order, samples, claim, units);
    *n_units = units.size();
    if (units.size() > cap) return bfail(nullptr, LAP_ERR_TOO_LARGE, "unit arrays too short");
    if (!unit_graph || !unit_first) return bfail(nullptr, LAP_ERR_INVALID_ARG, "unit arrays are NULL");
    for (size_t k = 0; k < units.size(); ++k) {
        unit_graph[k] = units[k].x;
        unit_first[k] = units[k].y;
    }
    return LAP_OK;
}

lap_status lap_batch_create(int32_t n_graphs, const int32_t *n, const int32_t *const *row_ptr,
                            const int32_t *const *col_idx, const int32_t *roots, lap_batch **out)
{
    if (!out) return bfail(nullptr, LAP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_graphs < 1 || n_graphs > 65535) return bfail(nullptr, LAP_ERR_INVALID_ARG, "n_graphs must be in [1, 65535]");
    if (!n || !row_ptr || !col_idx) return bfail(nullptr, LAP_ERR_INVALID_ARG, "n, row_ptr or col_idx is NULL");
    lap_batch *b = new (std::nothrow) lap_batch();
    if (!b) return bfail(nullptr, LAP_ERR_OOM, "host allocation failed");
    auto bad = [&](lap_status s, const std::string &m) {
        free_batch(b);
        delete b;
        return bfail(nullptr, s, m);
    };
    b->G = n_graphs;
    b->n.assign(n, n + n_graphs);
    b->roots.assign((size_t)n_graphs, -1);
    b->arcs.resize((size_t)n_graphs);
    b->node_off.resize((size_t)n_graphs + 1);
    b->arc_off.resize((size_t)n_graphs + 1);
    b->node_off[0] = b->arc_off[0] = 0;
    for (int32_t g = 0; g < n_graphs; ++g) {
        const std::string which = "graph " + std::to_string(g) + ": ";
        if (n[g] < 2) return bad(LAP_ERR_INVALID_ARG, which + "n must be at least 2");
        if (!row_ptr[g] || !col_idx[g]) return bad(LAP_ERR_INVALID_ARG, which + "row_ptr or col_idx is NULL");
        if (row_ptr[g][0] != 0 || row_ptr[g][n[g]] < 0) return bad(LAP_ERR_BAD_CSR, which + "row_ptr[0] must be 0 and row_ptr[n] >= 0");
        if (row_ptr[g][n[g]] == 0) return bad(LAP_ERR_DISCONNECTED, which + "graph has no edges");
        if (roots && roots[g] >= n[g]) return bad(LAP_ERR_INVALID_ARG, which + "root out of range");
        if (roots) b->roots[(size_t)g] = roots[g];
        b->arcs[(size_t)g] = row_ptr[g][n[g]];
        b->node_off[(size_t)g + 1] = b->node_off[(size_t)g] + n[g];
        b->arc_off[(size_t)g + 1] = b->arc_off[(size_t)g] + b->arcs[(size_t)g];
        b->max_n = std::max(b->max_n, n[g]);
    }
    b->total_n = b->node_off[(size_t)n_graphs];
    b->total_arcs = b->arc_off[(size_t)n_graphs];
    // Graphs passed with the same (n, row_ptr, col_idx) pointers share one copy
    // of the CSR (e.g. one graph sampled from many roots).
    b->src.resize((size_t)n_graphs);
    b->csr_node_off.resize((size_t)n_graphs);
    b->csr_arc_off.resize((size_t)n_graphs);
    for (int32_t g = 0; g < n_graphs; ++g) {
        int32_t same = g;
        for (int32_t h = 0; h < g && same == g; ++h)
            if (b->src[(size_t)h] == h && n[h] == n[g] && row_ptr[h] == row_ptr[g] && col_idx[h] == col_idx[g]) same = h;
        b->src[(size_t)g] = same;
        if (same == g) {
            b->csr_node_off[(size_t)g] = b->csr_nodes;
            b->csr_arc_off[(size_t)g] = b->csr_arcs;
            b->csr_nodes += n[g];
            b->csr_arcs += b->arcs[(size_t)g];
        } else {
            b->csr_node_off[(size_t)g] = b->csr_node_off[(size_t)same];
            b->csr_arc_off[(size_t)g] = b->csr_arc_off[(size_t)same];
        }
    }
    if (b->total_arcs >= (1ll << 40)) return bad(LAP_ERR_TOO_LARGE, "more than 2^40 arcs in the batch");
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
    if (b->num_sms <= 0) b->num_sms = 1;
    const size_t G = (size_t)n_graphs, tn = (size_t)b->total_n;
    int32_t *d_row_ptr = nullptr;
    bool ok = balloc(&d_row_ptr, (size_t)b->csr_nodes + G) == cudaSuccess &&
              balloc(&b->d_col, (size_t)b->csr_arcs) == cudaSuccess &&
              balloc(&b->d_rowinfo, (size_t)b->csr_nodes) == cudaSuccess && balloc(&b->d_rep1, tn) == cudaSuccess &&
              balloc(&b->d_cnt2, tn) == cudaSuccess && balloc(&b->d_ldiag, tn) == cudaSuccess &&
              balloc(&b->d_ecc, tn) == cudaSuccess && balloc(&b->d_scratch, (size_t)b->max_n) == cudaSuccess &&
              balloc(&b->d_red, G * 1026) == cudaSuccess && balloc(&b->d_graphs, G) == cudaSuccess &&
              balloc(&b->d_acc, G) == cudaSuccess && balloc(&b->d_done, G) == cudaSuccess &&
              balloc(&b->d_tdone, G) == cudaSuccess && balloc(&b->d_ctl, 1) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaFree(d_row_ptr);
        return bad(LAP_ERR_OOM, "device allocation failed");
    }
    auto cuda_bad = [&](cudaError_t e, const char *where) {
        cudaFree(d_row_ptr);
        return bad(LAP_ERR_CUDA, std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e));
    };
    cudaStream_t st = nullptr;
    cudaError_t e = cudaMemsetAsync(b->d_acc, 0, sizeof(LapDevAcc) * G, st);
    for (size_t g = 0; g < G && e == cudaSuccess; ++g) {
        if (b->src[g] != (int32_t)g) continue;
        int32_t *rp = d_row_ptr + b->csr_node_off[g] + (int64_t)g;
        e = cudaMemcpyAsync(rp, row_ptr[g], sizeof(int32_t) * ((size_t)n[g] + 1), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_col + b->csr_arc_off[g], col_idx[g], sizeof(int32_t) * (size_t)b->arcs[g],
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = lap_launch_validate(rp, b->d_col + b->csr_arc_off[g], n[g], b->arcs[g], &b->d_acc[g].status, st);
    }
    std::vector<LapDevAcc> acc(G);
    if (e == cudaSuccess) e = cudaMemcpyAsync(acc.data(), b->d_acc, sizeof(LapDevAcc) * G, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_bad(e, "batch ingest");
    for (size_t g = 0; g < G; ++g) {
        const std::string which = "graph " + std::to_string(g) + ": ";
        const unsigned int h = acc[g].status;
        lap_status s = LAP_OK;
        std::string m;
        if (h & LAP_DEV_BAD_CSR) { s = LAP_ERR_BAD_CSR; m = "CSR malformed: row_ptr not monotone, column out of range, or a row not strictly ascending"; }
        else if (h & LAP_DEV_SELF_LOOP) { s = LAP_ERR_SELF_LOOP; m = "graph has a self-loop"; }
        else if (h & LAP_DEV_NOT_SYMMETRIC) { s = LAP_ERR_NOT_SYMMETRIC; m = "CSR is not symmetric (graph must be undirected)"; }
        if (s != LAP_OK) {
            cudaFree(d_row_ptr);
            return bad(s, which + m);
        }
    }
    for (size_t g = 0; g < G && e == cudaSuccess; ++g)
        if (b->src[g] == (int32_t)g)
            e = lap_launch_rowinfo(d_row_ptr + b->csr_node_off[g] + (int64_t)g, n[g], b->d_rowinfo + b->csr_node_off[g], st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_row_ptr);
    d_row_ptr = nullptr;
    if (e != cudaSuccess) return cuda_bad(e, "row records");
    // Roots: the highest degree, smallest id on ties, where none was given.
    e = cudaMemsetAsync(b->d_tdone, 0, sizeof(unsigned long long) * G, st);
    for (size_t g = 0; g < G && e == cudaSuccess; ++g)
        if (b->roots[g] < 0) e = lap_launch_argmax_degree(b->d_rowinfo + b->csr_node_off[g], n[g], b->d_tdone + g, st);
    std::vector<unsigned long long> best(G);
    if (e == cudaSuccess) e = cudaMemcpyAsync(best.data(), b->d_tdone, sizeof(unsigned long long) * G, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_bad(e, "root selection");
    for (size_t g = 0; g < G; ++g)
        if (b->roots[g] < 0) b->roots[g] = (int32_t)(0xFFFFFFFFu - (uint32_t)(best[g] & 0xFFFFFFFFull));
    // Connectivity: level-synchronous BFS of all graphs together (hop
    // distances kept in the ldiag arena, which holds 8 bytes per node).
    int32_t *hops = reinterpret_cast<int32_t *>(b->d_ldiag);
    for (size_t g = 0; g < G && e == cudaSuccess; ++g)
        e = lap_launch_bfs_init(hops + b->node_off[g], n[g], b->roots[g], st);
    std::vector<int64_t> reached(G, 1);
    std::vector<char> active(G, 1);
    std::vector<unsigned int> found(G);
    for (int32_t level = 0; e == cudaSuccess; ++level) {
        e = cudaMemsetAsync(b->d_done, 0, sizeof(unsigned int) * G, st);
        bool any = false;
        for (size_t g = 0; g < G && e == cudaSuccess; ++g) {
            if (!active[g]) continue;
            any = true;
            e = lap_launch_bfs_level(b->d_rowinfo + b->csr_node_off[g], b->d_col + b->csr_arc_off[g], hops + b->node_off[g], n[g],
                                     level, b->d_done + g, st);
        }
        if (!any || e != cudaSuccess) break;
        e = cudaMemcpyAsync(found.data(), b->d_done, sizeof(unsigned int) * G, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        for (size_t g = 0; g < G && e == cudaSuccess; ++g) {
            if (!active[g]) continue;
            if (found[g] == 0) active[g] = 0;
            reached[g] += found[g];
        }
    }
    if (e != cudaSuccess) return cuda_bad(e, "connectivity check");
    for (size_t g = 0; g < G; ++g)
        if (reached[g] != n[g])
            return bad(LAP_ERR_DISCONNECTED, "graph " + std::to_string(g) + ": root " + std::to_string(b->roots[g]) +
                                                 " reaches " + std::to_string(reached[g]) + " of " + std::to_string(n[g]) +
                                                 " nodes: graph is not connected");
    b->h_graphs.resize(G);
    for (size_t g = 0; g < G; ++g) {
        LapBatchGraph &d = b->h_graphs[g];
        memset(&d, 0, sizeof(d));
        d.rowinfo = b->d_rowinfo + b->csr_node_off[g];
        d.col = b->d_col + b->csr_arc_off[g];
        d.rep1 = b->d_rep1 + b->node_off[g];
        d.cnt2 = b->d_cnt2 + b->node_off[g];
        d.ldiag = b->d_ldiag + b->node_off[g];
        d.ecc = b->d_ecc + b->node_off[g];
        d.arcs = b->arcs[g];
        d.step_limit = step_limit_of(n[g]);
        d.n = n[g];
        d.root = b->roots[g];
    }
    e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_bad(e, "creating the capture stream");
    *out = b;
    return LAP_OK;
}

lap_status lap_batch_destroy(lap_batch *b)
{
    if (!b) return LAP_OK;
    cudaStreamSynchronize(b->stream);
    free_batch(b);
    delete b;
    return LAP_OK;
}

lap_status lap_batch_set_stream(lap_batch *b, void *cuda_stream)
{
    if (!b) return bfail(nullptr, LAP_ERR_INVALID_ARG, "NULL handle");
    b->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    return LAP_OK;
}

lap_status lap_batch_set_option(lap_batch *b, int32_t option, int64_t value)
{
    if (!b) return bfail(nullptr, LAP_ERR_INVALID_ARG, "NULL handle");
    if (value < 0) return bfail(b, LAP_ERR_INVALID_ARG, "option value must be >= 0");
    switch (option) {
    case LAP_BOPT_LANES:
        b->lanes_opt = (uint64_t)value;
        return LAP_OK;
    case LAP_BOPT_CLAIM:
        if (value < 1 || value > 65536) return bfail(b, LAP_ERR_INVALID_ARG, "claim must be in [1, 65536]");
        b->claim_opt = (uint32_t)value;
        return LAP_OK;
    case LAP_BOPT_ORDER:
        if (value > 2) return bfail(b, LAP_ERR_INVALID_ARG, "order must be 0, 1 or 2");
        b->order_opt = (int)value;
        return LAP_OK;
    case LAP_BOPT_BLOCK:
        if (value != 0 && (value % 32 != 0 || value > 256)) return bfail(b, LAP_ERR_INVALID_ARG, "block must be 0 or a multiple of 32 up to 256");
        b->block_opt = (int)value;
        return LAP_OK;
    case LAP_BOPT_PATHS:
        if (value > 1) return bfail(b, LAP_ERR_INVALID_ARG, "paths must be 0 or 1");
        if (b->paths_opt != (uint32_t)value) b->meta_dirty = true;   // the slot layout changes
        b->paths_opt = (uint32_t)value;
        return LAP_OK;
    case LAP_BOPT_STACK:
        if (value != 0 && (value < 16 || value > (1 << 26) || (value & 3))) return bfail(b, LAP_ERR_INVALID_ARG, "stack capacity must be 0 or a multiple of 4 in [16, 2^26]");
        if ((uint32_t)value != b->stack_opt) b->meta_dirty = true;
        b->stack_opt = (uint32_t)value;
        return LAP_OK;
    default:
        return bfail(b, LAP_ERR_INVALID_ARG, "unknown option");
    }
}

lap_status lap_batch_workspace_query(const lap_batch *b, uint64_t lanes, uint64_t *bytes)
{
    if (!b || !bytes) return bfail(nullptr, LAP_ERR_INVALID_ARG, "NULL argument");
    *bytes = lanes * slot_bytes_of(b);
    return LAP_OK;
}

lap_status lap_batch_set_workspace(lap_batch *b, void *device_ptr, uint64_t bytes)
{
    if (!b) return bfail(nullptr, LAP_ERR_INVALID_ARG, "NULL handle");
    if (!device_ptr || (reinterpret_cast<uintptr_t>(device_ptr) & 255u)) return bfail(b, LAP_ERR_INVALID_ARG, "workspace must be non-NULL and 256-byte aligned");
    cudaStreamSynchronize(b->stream);
    if (b->ws_owned) cudaFree(b->ws);
    b->ws = device_ptr;
    b->ws_bytes = bytes & ~255ull;
    b->ws_owned = false;
    b->meta_dirty = true;
    b->key_valid = false;
    return LAP_OK;
}

lap_status lap_batch_run(lap_batch *b, uint64_t samples_per_graph, uint64_t seed)
{
    if (!b) return bfail(nullptr, LAP_ERR_INVALID_ARG, "NULL handle");
    if (b->sticky == LAP_ERR_CUDA) return b->sticky;
    if (samples_per_graph < 1 || samples_per_graph > (1ull << 31)) return bfail(b, LAP_ERR_INVALID_ARG, "samples_per_graph must be in [1, 2^31]");
    const uint64_t total = samples_per_graph * (uint64_t)b->G;
    if (total > (1ull << 32)) return bfail(b, LAP_ERR_TOO_LARGE, "at most 2^32 samples per run");
    b->sticky = LAP_OK;
    lap_status s = ensure_workspace(b);
    if (s != LAP_OK) return s;
    if (b->ovf_cap < total) {
        cudaFree(b->d_ovf);
        cudaFree(b->d_rerun_ids);
        b->d_ovf = nullptr;
        b->d_rerun_ids = nullptr;
        b->ovf_cap = 0;
        if (balloc(&b->d_ovf, (size_t)total) != cudaSuccess || balloc(&b->d_rerun_ids, (size_t)total) != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, LAP_ERR_OOM, "overflow list allocation failed");
        }
        b->ovf_cap = (uint32_t)std::min<uint64_t>(total, 0xFFFFFFFFull);
        b->key_valid = false;
    }
    int block = 0;
    const uint64_t lanes = lanes_for(b, samples_per_graph, b->lanes_opt, &block);
    if (lanes == 0) return bfail(b, LAP_ERR_OOM, "no lane fits the workspace");
    const uint32_t claim = b->claim_opt;
    if (!b->key_valid || !b->exec || b->key_samples != samples_per_graph || b->key_seed != seed || b->key_lanes != lanes ||
        b->key_claim != claim || b->key_order != b->order_opt || b->key_block != block || b->key_stack != stack_cap_of(b) ||
        b->key_paths != b->paths_opt) {
        s = capture(b, samples_per_graph, seed, lanes, claim, block);
        if (s != LAP_OK) return s;
    }
    B_CUDA(b, cudaGraphLaunch(b->exec, b->stream));
    b->omega = samples_per_graph;
    b->seed = seed;
    b->ran = true;
    b->checked = false;
    return LAP_OK;
}

lap_status lap_batch_sync(lap_batch *b) { return finish(b); }

lap_status lap_batch_autotune(lap_batch *b, uint64_t samples_per_graph, uint64_t seed, double window_ms,
                              int32_t max_trials, int64_t *trial_lanes, int32_t *trial_claim,
                              double *trial_steps_per_s, int32_t *n_trials)
{
    lap_status s = check_handle(b);
    if (s != LAP_OK && s != LAP_ERR_STEP_LIMIT) return s;
    if (samples_per_graph < 1 || samples_per_graph > (1ull << 31) || !(window_ms > 0.0) || window_ms > 60000.0)
        return bfail(b, LAP_ERR_INVALID_ARG, "bad autotune arguments");
    if (samples_per_graph * (uint64_t)b->G > (1ull << 32)) return bfail(b, LAP_ERR_TOO_LARGE, "at most 2^32 samples per run");
    if ((s = ensure_workspace(b)) != LAP_OK) return s;
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    const uint64_t lanes_max = lanes_for(b, samples_per_graph, 0, nullptr);
    if (lanes_max == 0) return bfail(b, LAP_ERR_OOM, "no lane fits the workspace");
    const uint32_t claim0 = b->claim_opt;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    B_CUDA(b, cudaEventCreate(&ev0));
    B_CUDA(b, cudaEventCreate(&ev1));
    int32_t rows = 0;
    auto probe = [&](uint64_t lanes, uint32_t claim, double *score) -> lap_status {
        lap_status r = upload_plan(b, samples_per_graph, claim);
        if (r != LAP_OK) return r;
        int block = b->block_opt > 0 ? b->block_opt : lap_pick_block(lanes, b->num_sms);
        LapBatchLaunch p = make_launch(b, seed, lanes, claim, block);
        p.window_ns = (unsigned long long)(window_ms * 1e6);
        double sum = 0.0;
        for (int k = 0; k < 3; ++k) {
            LapBatchCtl c;
            memset(&c, 0, sizeof(c));
            c.t0 = ~0ull;
            c.claim = (unsigned int)((uint64_t)b->n_units * (uint64_t)k / 3ull);
            B_CUDA(b, cudaMemcpyAsync(b->d_ctl, &c, sizeof(c), cudaMemcpyHostToDevice, b->stream));
            B_CUDA(b, cudaMemsetAsync(b->d_slot_meta, 0, sizeof(unsigned int) * b->meta_cap, b->stream));
            B_CUDA(b, cudaMemsetAsync(b->d_done, 0, sizeof(unsigned int) * (size_t)b->G, b->stream));
            B_CUDA(b, cudaEventRecord(ev0, b->stream));
            B_CUDA(b, lap_launch_batch(p, true, b->stream));
            B_CUDA(b, cudaEventRecord(ev1, b->stream));
            B_CUDA(b, cudaMemcpyAsync(&c, b->d_ctl, sizeof(c), cudaMemcpyDeviceToHost, b->stream));
            B_CUDA(b, cudaStreamSynchronize(b->stream));
            float ms = 0.f;
            B_CUDA(b, cudaEventElapsedTime(&ms, ev0, ev1));
            sum += (double)c.steps / (ms > 0.f ? ms * 1e-3 : 1e-3);
        }
        *score = sum / 3.0;
        if (rows < max_trials) {
            if (trial_lanes) trial_lanes[rows] = (int64_t)lanes;
            if (trial_claim) trial_claim[rows] = (int32_t)claim;
            if (trial_steps_per_s) trial_steps_per_s[rows] = *score;
        }
        ++rows;
        return LAP_OK;
    };
    uint64_t best_lanes = lanes_max;
    uint32_t best_claim = 1;
    double best = -1.0;
    for (int q = 1; q <= 4 && s == LAP_OK; ++q) {
        uint64_t l = lanes_max * (uint64_t)q / 4ull;
        l = l >= 32 ? l & ~31ull : l;
        if (l == 0) continue;
        double sc = 0.0;
        s = probe(l, 1, &sc);
        if (s == LAP_OK && sc > best) { best = sc; best_lanes = l; }
    }
    for (uint32_t c : {4u, 16u}) {
        if (s != LAP_OK) break;
        double sc = 0.0;
        s = probe(best_lanes, c, &sc);
        if (s == LAP_OK && sc > best) { best = sc; best_claim = c; }
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    b->meta_dirty = true;                    // probes stop lanes inside samples
    b->key_valid = false;                    // the descriptors and units were re-uploaded
    b->ran = false;                          // counts are scratch
    if (s != LAP_OK) {
        b->claim_opt = claim0;
        return s;
    }
    B_CUDA(b, cudaMemsetAsync(b->d_slot_meta, 0, sizeof(unsigned int) * b->meta_cap, b->stream));
    b->meta_dirty = false;
    b->lanes_opt = best_lanes;
    b->claim_opt = best_claim;
    if (n_trials) *n_trials = rows;
    return LAP_OK;
}

lap_status lap_batch_ecc(lap_batch *b, double *out, int on_device)
{
    lap_status s = finish(b);
    if (s != LAP_OK) return s;
    if (!out) return bfail(b, LAP_ERR_INVALID_ARG, "output pointer is NULL");
    B_CUDA(b, cudaMemcpyAsync(out, b->d_ecc, sizeof(double) * (size_t)b->total_n,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    return LAP_OK;
}

lap_status lap_batch_ldiag(lap_batch *b, double *out, int on_device)
{
    lap_status s = finish(b);
    if (s != LAP_OK) return s;
    if (!out) return bfail(b, LAP_ERR_INVALID_ARG, "output pointer is NULL");
    B_CUDA(b, cudaMemcpyAsync(out, b->d_ldiag, sizeof(double) * (size_t)b->total_n,
                              on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    return LAP_OK;
}

lap_status lap_batch_kemeny(lap_batch *b, double *out)
{
    lap_status s = finish(b);
    if (s != LAP_OK) return s;
    if (!out) return bfail(b, LAP_ERR_INVALID_ARG, "output pointer is NULL");
    std::vector<LapDevAcc> acc((size_t)b->G);
    B_CUDA(b, cudaMemcpyAsync(acc.data(), b->d_acc, sizeof(LapDevAcc) * acc.size(), cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    // Alg. 4 per graph: kappa = (sum Y1 - sum Y2) / omega.
    for (int32_t g = 0; g < b->G; ++g)
        out[g] = ((double)acc[(size_t)g].sum_y1 - (double)acc[(size_t)g].sum_y2) / (double)b->omega;
    return LAP_OK;
}

lap_status lap_batch_kirchhoff(lap_batch *b, double *out)
{
    lap_status s = finish(b);
    if (s != LAP_OK) return s;
    if (!out) return bfail(b, LAP_ERR_INVALID_ARG, "output pointer is NULL");
    // The batched finalize leaves graph g's Tr(L^+) at red[g * 1026 + 1025].
    B_CUDA(b, cudaMemcpy2DAsync(out, sizeof(double), b->d_red + 1025, sizeof(double) * 1026, sizeof(double),
                                (size_t)b->G, cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    return LAP_OK;
}

lap_status lap_batch_completion(lap_batch *b, double *seconds)
{
    lap_status s = finish(b);
    if (s != LAP_OK) return s;
    if (!seconds) return bfail(b, LAP_ERR_INVALID_ARG, "output pointer is NULL");
    std::vector<unsigned long long> t((size_t)b->G);
    LapBatchCtl c;
    B_CUDA(b, cudaMemcpyAsync(t.data(), b->d_tdone, sizeof(unsigned long long) * t.size(), cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(b, cudaMemcpyAsync(&c, b->d_ctl, sizeof(c), cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    for (int32_t g = 0; g < b->G; ++g)
        seconds[g] = t[(size_t)g] >= c.t0 ? (double)(t[(size_t)g] - c.t0) * 1e-9 : 0.0;
    return LAP_OK;
}

lap_status lap_batch_counts(lap_batch *b, int32_t graph, uint64_t *cnt1, uint64_t *cnt2, uint64_t *sums, int on_device)
{
    lap_status s = finish(b);
    if (s != LAP_OK) return s;
    if (graph < 0 || graph >= b->G) return bfail(b, LAP_ERR_INVALID_ARG, "graph index out of range");
    const LapBatchGraph &d = b->h_graphs[(size_t)graph];
    const size_t bytes = sizeof(uint64_t) * (size_t)d.n;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (cnt1) {
        B_CUDA(b, lap_launch_counts(d.n, d.root, b->omega, d.rep1, b->d_scratch, b->stream));
        B_CUDA(b, cudaMemcpyAsync(cnt1, b->d_scratch, bytes, kind, b->stream));
    }
    if (cnt2) B_CUDA(b, cudaMemcpyAsync(cnt2, d.cnt2, bytes, kind, b->stream));
    if (sums) {
        LapDevAcc h;
        B_CUDA(b, cudaMemcpyAsync(&h, b->d_acc + graph, sizeof(h), cudaMemcpyDeviceToHost, b->stream));
        B_CUDA(b, cudaStreamSynchronize(b->stream));
        sums[0] = b->omega;
        sums[1] = h.sum_y1;
        sums[2] = h.sum_y2;
        sums[3] = b->seed;
    }
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    return LAP_OK;
}

lap_status lap_batch_set_path_start(lap_batch *b, int32_t graph, int32_t start)
{
    if (!b) return bfail(nullptr, LAP_ERR_INVALID_ARG, "NULL handle");
    if (graph < 0 || graph >= b->G) return bfail(b, LAP_ERR_INVALID_ARG, "graph index out of range");
    LapBatchGraph &d = b->h_graphs[(size_t)graph];
    if (start < -1 || start >= d.n) return bfail(b, LAP_ERR_INVALID_ARG, "path start must be -1 or a node id of the graph");
    d.ustart = start >= 0 ? (uint32_t)start + 1u : 0u;
    // The kernels read the descriptors at run time: update the device copy.
    B_CUDA(b, cudaMemcpyAsync(b->d_graphs + graph, &d, sizeof(d), cudaMemcpyHostToDevice, b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    return LAP_OK;
}

lap_status lap_batch_lv_row(lap_batch *b, int32_t graph, double *out, int on_device)
{
    lap_status s = finish(b);
    if (s != LAP_OK) return s;
    if (graph < 0 || graph >= b->G) return bfail(b, LAP_ERR_INVALID_ARG, "graph index out of range");
    if (!out) return bfail(b, LAP_ERR_INVALID_ARG, "output pointer is NULL");
    const LapBatchGraph &d = b->h_graphs[(size_t)graph];
    double *dst = on_device ? out : reinterpret_cast<double *>(b->d_scratch);
    B_CUDA(b, lap_launch_lv_row(d.rowinfo, d.n, b->omega, d.cnt2, dst, b->stream));
    if (!on_device)
        B_CUDA(b, cudaMemcpyAsync(out, dst, sizeof(double) * (size_t)d.n, cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    return LAP_OK;
}

lap_status lap_batch_graph_info(const lap_batch *b, int32_t graph, int32_t *n, int64_t *arcs, int32_t *root,
                                int64_t *offset)
{
    if (!b) return bfail(nullptr, LAP_ERR_INVALID_ARG, "NULL handle");
    if (graph < 0 || graph >= b->G) return LAP_ERR_INVALID_ARG;
    if (n) *n = b->n[(size_t)graph];
    if (arcs) *arcs = b->arcs[(size_t)graph];
    if (root) *root = b->roots[(size_t)graph];
    if (offset) *offset = b->node_off[(size_t)graph];
    return LAP_OK;
}

lap_status lap_batch_stat(const lap_batch *b, int32_t which, int64_t *value)
{
    if (!b || !value) return bfail(nullptr, LAP_ERR_INVALID_ARG, "NULL argument");
    switch (which) {
    case LAP_BSTAT_LANES: *value = (int64_t)(b->ws ? lanes_for(b, b->omega ? b->omega : 1ull << 31, b->lanes_opt, nullptr) : 0); return LAP_OK;
    case LAP_BSTAT_CLAIM: *value = b->claim_opt; return LAP_OK;
    case LAP_BSTAT_UNITS: *value = b->n_units; return LAP_OK;
    case LAP_BSTAT_RERUNS: *value = b->reruns; return LAP_OK;
    case LAP_BSTAT_GRAPH_CAPTURES: *value = b->captures; return LAP_OK;
    default: return LAP_ERR_INVALID_ARG;
    }
}

}  // extern "C"
