// Host side of the C ABI declared in include/lap.h: argument checks, device
// memory of a handle, stream handling, launch sizing and error reporting.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lap_internal.h"

namespace {

thread_local std::string g_create_error = "no error";

lap_status fail(lap_graph *g, lap_status s, const std::string &msg)
{
    if (g) g->err = msg;
    else g_create_error = msg;
    return s;
}

lap_status cuda_fail(lap_graph *g, cudaError_t e, const char *where)
{
    std::string m = std::string("CUDA error in ") + where + ": " + cudaGetErrorString(e);
    if (g) g->sticky = LAP_ERR_CUDA;
    return fail(g, LAP_ERR_CUDA, m);
}

#define LAP_CUDA(g, call)                                            \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail((g), e_, #call);     \
    } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t count)
{
    return cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (count > 0 ? count : 1));
}

void free_all(lap_graph *g)
{
    cudaFree(g->d_row_ptr);
    cudaFree(g->d_col);
    cudaFree(g->d_rowinfo);
    cudaFree(g->d_hops);
    cudaFree(g->d_rep1);
    cudaFree(g->d_cnt2);
    cudaFree(g->d_acc);
    cudaFree(g->d_ldiag);
    cudaFree(g->d_ecc);
    cudaFree(g->d_red);
    cudaFree(g->d_aux);
    cudaFree(g->d_slot_epoch);
    cudaFree(g->d_ovf_ids);
    cudaFree(g->d_cv_h1);
    cudaFree(g->d_cv_S1);
    cudaFree(g->d_cv_h2);
    cudaFree(g->d_cv_S2);
    cudaFree(g->d_cv_a1);
    cudaFree(g->d_cv_a2);
    cudaFree(g->d_cv_p2);
    cudaFree(g->d_feat_scratch);
    cudaFree(g->d_bpar);
    cudaFree(g->d_st_x1);
    cudaFree(g->d_st_x2);
    cudaFree(g->d_st_x2d);
    cudaFree(g->d_st_rep1);
    cudaFree(g->d_st_ldiag);
    cudaFree(g->d_st_ecc);
    cudaFree(g->d_st_red);
    cudaFree(g->d_st_acc);
    cudaFree(g->d_st_scratch);
    if (g->ws_owned) cudaFree(g->ws);
}

lap_status check_sticky(lap_graph *g)
{
    if (!g) return fail(nullptr, LAP_ERR_INVALID_ARG, "NULL handle");
    if (g->sticky != LAP_OK) return g->sticky;
    return LAP_OK;
}

uint64_t default_step_limit(int32_t n) { return (1ull << 20) + 1024ull * (uint64_t)n; }

uint64_t n_pad_of(const lap_graph *g) { return ((uint64_t)g->n + 255ull) & ~255ull; }

// Loop-erased paths of a Wilson run on small-world graphs grow like sqrt(n)
// (about 1.6e3 nodes at most at n = 1e6 with a hub root), so the default
// stack holds 16 sqrt(n) entries, at least 1024.
uint32_t stack_cap_of(const lap_graph *g)
{
    if (g->stack_cap) return g->stack_cap;
    uint64_t c = 1024;
    while (c * c < 256ull * (uint64_t)g->n && c < (1u << 20)) c <<= 1;
    return (uint32_t)c;
}

uint64_t slot_bytes_of(const lap_graph *g, int kernel)
{
    if (kernel == LAP_KERNEL_WIDE) return 8ull * (uint64_t)g->n;
    if (kernel == LAP_KERNEL_GROUP)
        // Control block, 16-bit words, departure bytes of the two loop-included
        // paths (2 per node, LAP_OPT_PATHS only), path stacks: 8 stacks' worth
        // of entries shared out among the sample's walkers.
        return (64ull + (g->paths_opt ? 4ull : 2ull) * n_pad_of(g) + 4ull * stack_cap_of(g) * 8ull + 255ull) & ~255ull;
    // State bytes, path-count bytes (loop-included paths only), stack, count table.
    return ((g->paths_opt ? 2ull : 1ull) * n_pad_of(g) + 4ull * stack_cap_of(g) + (8ull << lap_table_log2(g->n)) +
            255ull) & ~255ull;
}

// Kernel 3 covers every estimator form (own absorbed walks or loop-included
// paths, with or without the control variate) on graphs with n < 2^22 (its
// stack entries hold 22-bit node ids).
bool group_ok(const lap_graph *g)
{
    return g->n < (1 << 22) && !g->compact_disabled &&
           (!g->ws || g->ws_bytes >= slot_bytes_of(g, LAP_KERNEL_GROUP));
}

// Calls of at most this many samples per SM take kernel 3 automatically:
// below it one lane per sample leaves the GPU short of independent memory
// chains.  Measured on one GB300: on Barabasi-Albert 10^6, whose graph stays
// in L2, kernel 3 is ahead up to 32,768 samples and level at 65,536; on R-MAT
// scale 22, whose column array misses L2, it is ahead at 65,536 too.
constexpr uint64_t kGroupAutoPerSm = 320;
constexpr uint64_t kGroupAutoPerSmLarge = 1024;     // graphs whose arrays exceed kL2Graph
constexpr uint64_t kL2Graph = 96ull << 20;
// Smaller graphs keep kernel 2: on a 1000-node graph a Wilson run is ~1,600
// steps and a group's per-sample costs (slot clearing, chunk scans, walkers
// meeting on few nodes) outweigh the shorter runs (92,682 samples: 15.7 ms
// with kernel 2, 44 ms with 8 walkers; 23,170 samples with loop-included
// paths: 16 ms and 27 ms), while from 10^5 nodes up kernel 3 wins for small
// calls.  The threshold lies between the measured sizes.
constexpr int32_t kGroupAutoMinNodes = 1 << 14;

// Walkers per sample of kernel 3 for a call of n_samples: the option, or
// 16 when the call's 16 lanes per sample fit on the GPU at once (1280 lanes
// per SM: 5 blocks of 256), which halves a sample's time; else 8.
int walkers_for(const lap_graph *g, uint64_t n_samples)
{
    if (g->walkers) return g->walkers;
    return n_samples > 0 && n_samples * 16ull <= 1280ull * (uint64_t)g->num_sms ? 16 : 8;
}

// n_samples: the size of the call (0: a call large enough for kernel 2).
int choose_kernel(const lap_graph *g, uint64_t n_samples = 0)
{
    if (g->kernel_opt == LAP_KERNEL_WIDE) return LAP_KERNEL_WIDE;
    if (g->kernel_opt == LAP_KERNEL_GROUP && group_ok(g)) return LAP_KERNEL_GROUP;
    const bool large_graph = 4ull * (uint64_t)g->arcs + 8ull * (uint64_t)g->n > kL2Graph;
    const uint64_t per_sm = large_graph ? kGroupAutoPerSmLarge : kGroupAutoPerSm;
    if (g->kernel_opt == 0 && n_samples > 0 && n_samples <= per_sm * (uint64_t)g->num_sms &&
        g->n >= kGroupAutoMinNodes && group_ok(g))
        return LAP_KERNEL_GROUP;
    if (g->n >= (1 << 27) || g->compact_disabled) return LAP_KERNEL_WIDE;
    if (g->ws && g->ws_bytes < slot_bytes_of(g, LAP_KERNEL_COMPACT)) return LAP_KERNEL_WIDE;
    return LAP_KERNEL_COMPACT;
}

// Makes sure a workspace exists and holds the layout of `kernel`, zeroed
// when the layout changed (epoch bits then read "stale" everywhere).
lap_status ensure_workspace(lap_graph *g, int kernel)
{
    const uint64_t per_slot = slot_bytes_of(g, kernel);
    if (!g->ws) {
        size_t free_b = 0, total_b = 0;
        LAP_CUDA(g, cudaMemGetInfo(&free_b, &total_b));
        uint64_t want = (uint64_t)free_b / 2;
        uint64_t cap = per_slot * (uint64_t)g->num_sms * 2048ull;
        if (want > cap) want = cap;
        want = (want / 256) * 256;
        if (want < per_slot) return fail(g, LAP_ERR_OOM, "not enough device memory for one Wilson state");
        cudaError_t e = cudaMalloc(&g->ws, want);
        if (e != cudaSuccess) { cudaGetLastError(); g->ws = nullptr; return fail(g, LAP_ERR_OOM, "workspace allocation failed"); }
        g->ws_bytes = want;
        g->ws_owned = true;
        g->ws_zeroed = false;
    }
    const uint64_t slots = g->ws_bytes / per_slot;
    if (slots == 0) return fail(g, LAP_ERR_OOM, "workspace smaller than one sample's state");
    if (kernel == LAP_KERNEL_GROUP) {
        // Kernel 3 clears a slot at each sample start; the next kernel of
        // another layout zeroes the workspace again.
        g->last_kernel = kernel;
        g->ws_zeroed = false;
        return LAP_OK;
    }
    if (slots > g->slot_epoch_cap) {
        cudaFree(g->d_slot_epoch);
        g->d_slot_epoch = nullptr;
        g->slot_epoch_cap = 0;
        if (dalloc(&g->d_slot_epoch, slots) != cudaSuccess) { cudaGetLastError(); return fail(g, LAP_ERR_OOM, "slot table allocation failed"); }
        g->slot_epoch_cap = slots;
        g->ws_zeroed = false;
    }
    if (g->last_kernel != kernel) g->ws_zeroed = false;
    if (!g->ws_zeroed) {
        LAP_CUDA(g, cudaMemsetAsync(g->ws, 0, g->ws_bytes, g->stream));
        LAP_CUDA(g, cudaMemsetAsync(g->d_slot_epoch, 0, sizeof(unsigned int) * g->slot_epoch_cap, g->stream));
        g->ws_zeroed = true;
        g->last_kernel = kernel;
    }
    return LAP_OK;
}

uint64_t slots_for(const lap_graph *g, int kernel, uint64_t n_samples)
{
    uint64_t slots = g->ws ? g->ws_bytes / slot_bytes_of(g, kernel) : 0;
    if (g->slots_opt && g->slots_opt < slots) slots = g->slots_opt;
    if (n_samples && slots > n_samples) slots = n_samples;
    return slots;
}

lap_status launch(lap_graph *g, LapSampleLaunch &p, int kernel)
{
    p.slots = slots_for(g, kernel, p.count);
    p.slot_bytes = slot_bytes_of(g, kernel);
    p.n_pad = n_pad_of(g);
    p.tbl_log2 = lap_table_log2(g->n);
    p.stack_cap = kernel == LAP_KERNEL_COMPACT
                      ? (uint32_t)((p.slot_bytes - (p.paths ? 2ull : 1ull) * p.n_pad - (8ull << p.tbl_log2)) / 4ull)
                  : kernel == LAP_KERNEL_GROUP
                      ? (uint32_t)(((p.slot_bytes - 64ull - (p.paths ? 4ull : 2ull) * p.n_pad) / 4ull /
                                    (uint64_t)walkers_for(g, p.count)) & ~3ull)
                      : 0u;
    LAP_CUDA(g, cudaMemsetAsync(&g->d_acc->claim, 0, sizeof(unsigned int), g->stream));
    const cudaError_t e = kernel == LAP_KERNEL_WIDE    ? lap_launch_sample(p, g->stream)
                          : kernel == LAP_KERNEL_GROUP ? lap_launch_sample_group(p, walkers_for(g, p.count), g->stream)
                                                       : lap_launch_sample_compact(p, g->stream);
    if (e != cudaSuccess) {
        char buf[256];
        snprintf(buf, sizeof(buf), "sampler launch (kernel %d, %llu lanes, block %d, cv %d): %s", kernel,
                 (unsigned long long)p.slots, p.block > 0 ? p.block : lap_pick_block(p.slots, p.num_sms),
                 (p.cv_h1 || p.cv_h2) ? 1 : 0, cudaGetErrorString(e));
        g->sticky = LAP_ERR_CUDA;
        return fail(g, LAP_ERR_CUDA, buf);
    }
    return LAP_OK;
}

// Finishes a compact launch: the samples it withdrew (state did not fit one
// byte per node, see sampler_compact.cu) are re-run with the 8-byte kernel,
// which gives them exactly the counts the compact kernel would have.
lap_status resolve_pending(lap_graph *g)
{
    if (!g->pending) return LAP_OK;
    g->pending = false;
    LapDevAcc h;
    LAP_CUDA(g, cudaMemcpyAsync(&h, g->d_acc, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    if (h.ovf_count == 0) return LAP_OK;
    LAP_CUDA(g, cudaMemsetAsync(&g->d_acc->ovf_count, 0, sizeof(unsigned int), g->stream));
    g->fallbacks += h.ovf_count;
    lap_status s = ensure_workspace(g, LAP_KERNEL_WIDE);
    if (s != LAP_OK) return s;
    LapSampleLaunch p = g->pending_launch;
    // The workspace and the slot table are those ensure_workspace just set
    // up for the 8-byte layout (the table may have been (re)allocated).
    p.ws = g->ws;
    p.slot_epoch = g->d_slot_epoch;
    p.ids = g->d_ovf_ids;
    p.trace_base = p.first;
    p.count = h.ovf_count;
    return launch(g, p, LAP_KERNEL_WIDE);
}

// Reads the device status word and turns it into a sticky error.
lap_status poll_status(lap_graph *g)
{
    lap_status s = resolve_pending(g);
    if (s != LAP_OK) return s;
    LapDevAcc h;
    LAP_CUDA(g, cudaMemcpyAsync(&h, g->d_acc, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    if (h.status & LAP_DEV_STEP_LIMIT) {
        g->sticky = LAP_ERR_STEP_LIMIT;
        return fail(g, LAP_ERR_STEP_LIMIT, "a sample exceeded the per-sample step budget (LAP_OPT_STEP_LIMIT)");
    }
    if (h.status & LAP_DEV_K_OVERFLOW) {
        g->sticky = LAP_ERR_STEP_LIMIT;
        return fail(g, LAP_ERR_STEP_LIMIT, "a node was visited more than 2^30 times in one sample");
    }
    if (h.status & LAP_DEV_BAD_INDEX) {
        char buf[160];
        snprintf(buf, sizeof(buf), "internal error: node index out of range caught in the sampler (%llx)",
                 (unsigned long long)h.pad[0]);
        g->sticky = LAP_ERR_CUDA;
        return fail(g, LAP_ERR_CUDA, buf);
    }
    return LAP_OK;
}

// Process-wide choice of the MLP kernel (lap_mlp_select).
std::atomic<int32_t> g_mlp_kernel{LAP_MLP_TCGEN05};

cudaError_t launch_mlp(const float *P, const float *X, const float *T, int64_t n, float wk0, float wk1, float *Y,
                       float *G, float *loss, cudaStream_t st)
{
    return g_mlp_kernel.load() == LAP_MLP_MMA_SYNC ? lap_launch_mlp_mma_sync(P, X, T, n, wk0, wk1, Y, G, loss, st)
                                                   : lap_launch_mlp_tc(P, X, T, n, wk0, wk1, Y, G, loss, st);
}

}  // namespace

extern "C" {

int32_t lap_version(void) { return 10000; }

const char *lap_last_error(const lap_graph *g) { return g ? g->err.c_str() : g_create_error.c_str(); }

lap_status lap_graph_create(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int ptrs_on_device,
                            lap_graph **out)
{
    if (!out) return fail(nullptr, LAP_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 2) return fail(nullptr, LAP_ERR_INVALID_ARG, "n must be at least 2");
    if (!row_ptr || !col_idx) return fail(nullptr, LAP_ERR_INVALID_ARG, "row_ptr or col_idx is NULL");
    if (ptrs_on_device != 0 && ptrs_on_device != 1) return fail(nullptr, LAP_ERR_INVALID_ARG, "ptrs_on_device must be 0 or 1");

    int32_t first = 0, last = 0;
    if (ptrs_on_device) {
        cudaError_t e = cudaMemcpy(&first, row_ptr, sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(&last, row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "reading row_ptr ends");
    } else {
        first = row_ptr[0];
        last = row_ptr[n];
    }
    if (first != 0 || last < 0) return fail(nullptr, LAP_ERR_BAD_CSR, "row_ptr[0] must be 0 and row_ptr[n] >= 0");
    if (last == 0) return fail(nullptr, LAP_ERR_DISCONNECTED, "graph has no edges");

    lap_graph *g = new (std::nothrow) lap_graph();
    if (!g) return fail(nullptr, LAP_ERR_OOM, "host allocation failed");
    g->n = n;
    g->arcs = last;
    cudaGetDevice(&g->device);
    cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (g->num_sms <= 0) g->num_sms = 1;

    const size_t nn = (size_t)n;
    bool ok = dalloc(&g->d_row_ptr, nn + 1) == cudaSuccess && dalloc(&g->d_col, (size_t)last) == cudaSuccess &&
              dalloc(&g->d_rowinfo, nn) == cudaSuccess && dalloc(&g->d_hops, nn) == cudaSuccess &&
              dalloc(&g->d_rep1, nn) == cudaSuccess && dalloc(&g->d_cnt2, nn) == cudaSuccess &&
              dalloc(&g->d_acc, 1) == cudaSuccess && dalloc(&g->d_ldiag, nn) == cudaSuccess &&
              dalloc(&g->d_ecc, nn) == cudaSuccess && dalloc(&g->d_red, 1024 + 16) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_all(g);
        delete g;
        return fail(nullptr, LAP_ERR_OOM, "device allocation failed");
    }
    cudaMemcpyKind kind = ptrs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaError_t e = cudaMemcpyAsync(g->d_row_ptr, row_ptr, sizeof(int32_t) * (nn + 1), kind, g->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->d_col, col_idx, sizeof(int32_t) * (size_t)last, kind, g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_acc, 0, sizeof(LapDevAcc), g->stream);
    if (e == cudaSuccess) e = lap_launch_validate(g->d_row_ptr, g->d_col, n, last, &g->d_acc->status, g->stream);
    LapDevAcc h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, g->d_acc, sizeof(h), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        lap_status s = cuda_fail(nullptr, e, "graph ingest");
        free_all(g);
        delete g;
        return s;
    }
    lap_status bad = LAP_OK;
    if (h.status & LAP_DEV_BAD_CSR) bad = fail(nullptr, LAP_ERR_BAD_CSR, "CSR malformed: row_ptr not monotone, column out of range, or a row not strictly ascending");
    else if (h.status & LAP_DEV_SELF_LOOP) bad = fail(nullptr, LAP_ERR_SELF_LOOP, "graph has a self-loop");
    else if (h.status & LAP_DEV_NOT_SYMMETRIC) bad = fail(nullptr, LAP_ERR_NOT_SYMMETRIC, "CSR is not symmetric (graph must be undirected)");
    if (bad != LAP_OK) {
        free_all(g);
        delete g;
        return bad;
    }
    e = lap_launch_rowinfo(g->d_row_ptr, n, g->d_rowinfo, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) {
        lap_status s = cuda_fail(nullptr, e, "row records");
        free_all(g);
        delete g;
        return s;
    }
    g->err = "no error";
    *out = g;
    return LAP_OK;
}

lap_status lap_graph_destroy(lap_graph *g)
{
    if (!g) return LAP_OK;
    cudaStreamSynchronize(g->stream);
    free_all(g);
    delete g;
    return LAP_OK;
}

lap_status lap_set_stream(lap_graph *g, void *cuda_stream)
{
    if (!g) return fail(nullptr, LAP_ERR_INVALID_ARG, "NULL handle");
    g->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    return LAP_OK;
}

lap_status lap_set_option(lap_graph *g, int32_t option, int64_t value)
{
    if (!g) return fail(nullptr, LAP_ERR_INVALID_ARG, "NULL handle");
    if (value < 0 && !(option == LAP_OPT_PATH_START && value == -1))
        return fail(g, LAP_ERR_INVALID_ARG, "option value must be >= 0");
    switch (option) {
    case LAP_OPT_STEP_LIMIT:
        g->step_limit = value > (int64_t)(1ull << 62) ? (1ull << 62) : (uint64_t)value;
        return LAP_OK;
    case LAP_OPT_SLOTS:
        g->slots_opt = (uint64_t)value;
        return LAP_OK;
    case LAP_OPT_CURSOR:
        if (g->omega != 0) return fail(g, LAP_ERR_INVALID_ARG, "the cursor can only be set before the first sample after lap_set_root");
        if ((uint64_t)value >= (1ull << 32)) return fail(g, LAP_ERR_TOO_LARGE, "sample ids are limited to 2^32");
        g->cursor = (uint64_t)value;
        return LAP_OK;
    case LAP_OPT_WALKERS:
        if (value != 0 && value != 2 && value != 4 && value != 8 && value != 16)
            return fail(g, LAP_ERR_INVALID_ARG, "walkers must be 0 (automatic), 2, 4, 8 or 16");
        g->walkers = (int)value;
        return LAP_OK;
    case LAP_OPT_KERNEL:
        if (value > 3) return fail(g, LAP_ERR_INVALID_ARG, "kernel must be 0, 1, 2 or 3");
        if (value == LAP_KERNEL_GROUP && g->n >= (1 << 22)) return fail(g, LAP_ERR_INVALID_ARG, "kernel 3 needs n < 2^22");
        if (value == LAP_KERNEL_COMPACT && g->n >= (1 << 27)) return fail(g, LAP_ERR_INVALID_ARG, "kernel 2 needs n < 2^27");
        g->kernel_opt = (int)value;
        return LAP_OK;
    case LAP_OPT_STACK:
        if (value != 0 && (value < 16 || value > (1 << 22))) return fail(g, LAP_ERR_INVALID_ARG, "stack capacity must be 0 or in [16, 2^22]");
        g->stack_cap = (uint32_t)value;
        g->last_kernel = 0;
        return LAP_OK;
    case LAP_OPT_BLOCK:
        if (value != 0 && (value % 32 != 0 || value > 256)) return fail(g, LAP_ERR_INVALID_ARG, "block must be 0 or a multiple of 32 up to 256");
        g->block_opt = (int)value;
        return LAP_OK;
    case LAP_OPT_PATHS:
        if (value > 1) return fail(g, LAP_ERR_INVALID_ARG, "paths must be 0 or 1");
        if (g->omega != 0) return fail(g, LAP_ERR_INVALID_ARG, "the walk mode can only be set before the first sample after lap_set_root");
        if (g->paths_opt != (uint32_t)value) g->last_kernel = 0;     // the slot layout changes
        g->paths_opt = (uint32_t)value;
        return LAP_OK;
    case LAP_OPT_PATH_START:
        if (value >= g->n) return fail(g, LAP_ERR_INVALID_ARG, "path start must be -1 or a node id");
        if (g->omega != 0) return fail(g, LAP_ERR_INVALID_ARG, "the walk start can only be set before the first sample after lap_set_root");
        g->path_start = (int32_t)value;
        return LAP_OK;
    default:
        return fail(g, LAP_ERR_INVALID_ARG, "unknown option");
    }
}

lap_status lap_workspace_query(const lap_graph *g, uint64_t slots, uint64_t *bytes)
{
    if (!g || !bytes) return fail(nullptr, LAP_ERR_INVALID_ARG, "NULL argument");
    *bytes = slot_bytes_of(g, choose_kernel(g)) * slots;
    return LAP_OK;
}

lap_status lap_get_stat(lap_graph *g, int32_t stat, int64_t *value)
{
    if (!g || !value) return fail(nullptr, LAP_ERR_INVALID_ARG, "NULL argument");
    switch (stat) {
    case LAP_STAT_SLOTS: *value = (int64_t)slots_for(g, choose_kernel(g), 0); return LAP_OK;
    case LAP_STAT_KERNEL: *value = choose_kernel(g); return LAP_OK;
    case LAP_STAT_LAST_KERNEL: *value = g->used_kernel; return LAP_OK;
    case LAP_STAT_FALLBACKS: {
        lap_status s = resolve_pending(g);
        if (s != LAP_OK) return s;
        *value = g->fallbacks;
        return LAP_OK;
    }
    default: return fail(g, LAP_ERR_INVALID_ARG, "unknown statistic");
    }
}

lap_status lap_set_workspace(lap_graph *g, void *device_ptr, uint64_t bytes)
{
    if (!g) return fail(nullptr, LAP_ERR_INVALID_ARG, "NULL handle");
    if (!device_ptr || bytes < slot_bytes_of(g, LAP_KERNEL_WIDE)) return fail(g, LAP_ERR_INVALID_ARG, "workspace must hold at least 8*n bytes");
    if (reinterpret_cast<uintptr_t>(device_ptr) % 256 != 0) return fail(g, LAP_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    cudaStreamSynchronize(g->stream);
    if (g->ws_owned) cudaFree(g->ws);
    g->ws = device_ptr;
    g->ws_bytes = bytes & ~255ull;
    g->ws_owned = false;
    g->ws_zeroed = false;
    g->last_kernel = 0;
    return LAP_OK;
}

lap_status lap_set_root(lap_graph *g, int32_t v, int32_t *root_out)
{
    if (!g) return fail(nullptr, LAP_ERR_INVALID_ARG, "NULL handle");
    if (v >= g->n) return fail(g, LAP_ERR_INVALID_ARG, "root out of range");
    g->sticky = LAP_OK;
    g->root = -1;
    if (v < 0) {
        unsigned long long *best = reinterpret_cast<unsigned long long *>(g->d_red);
        LAP_CUDA(g, cudaMemsetAsync(best, 0, sizeof(unsigned long long), g->stream));
        LAP_CUDA(g, lap_launch_argmax_degree(g->d_rowinfo, g->n, best, g->stream));
        unsigned long long h = 0;
        LAP_CUDA(g, cudaMemcpyAsync(&h, best, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
        LAP_CUDA(g, cudaStreamSynchronize(g->stream));
        v = (int32_t)(0xFFFFFFFFu - (uint32_t)(h & 0xFFFFFFFFull));
    }
    // Breadth-first search from v: connectivity check and hop distances.
    unsigned int *found = reinterpret_cast<unsigned int *>(g->d_red);
    LAP_CUDA(g, lap_launch_bfs_init(g->d_hops, g->n, v, g->stream));
    int64_t reached = 1;
    for (int32_t level = 0;; ++level) {
        LAP_CUDA(g, cudaMemsetAsync(found, 0, sizeof(unsigned int), g->stream));
        LAP_CUDA(g, lap_launch_bfs_level(g->d_rowinfo, g->d_col, g->d_hops, g->n, level, found, g->stream));
        unsigned int h = 0;
        LAP_CUDA(g, cudaMemcpyAsync(&h, found, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
        LAP_CUDA(g, cudaStreamSynchronize(g->stream));
        if (h == 0) break;
        reached += h;
    }
    if (reached != g->n) {
        char buf[160];
        snprintf(buf, sizeof(buf), "root %d reaches %lld of %d nodes: graph is not connected", v, (long long)reached, g->n);
        return fail(g, LAP_ERR_DISCONNECTED, buf);
    }
    LAP_CUDA(g, cudaMemsetAsync(g->d_rep1, 0, sizeof(unsigned long long) * (size_t)g->n, g->stream));
    LAP_CUDA(g, cudaMemsetAsync(g->d_cnt2, 0, sizeof(unsigned long long) * (size_t)g->n, g->stream));
    LAP_CUDA(g, cudaMemsetAsync(g->d_acc, 0, sizeof(LapDevAcc), g->stream));
    if (g->d_cv_a1) {
        const size_t nb = sizeof(unsigned long long) * (size_t)g->n;
        LAP_CUDA(g, cudaMemsetAsync(g->d_cv_a1, 0, nb, g->stream));
        LAP_CUDA(g, cudaMemsetAsync(g->d_cv_a2, 0, nb, g->stream));
        LAP_CUDA(g, cudaMemsetAsync(g->d_cv_p2, 0, nb, g->stream));
    }
    if (g->d_st_x1) {
        const size_t nb = sizeof(unsigned long long) * (size_t)g->n;
        LAP_CUDA(g, cudaMemsetAsync(g->d_st_x1, 0, nb, g->stream));
        LAP_CUDA(g, cudaMemsetAsync(g->d_st_x2, 0, nb, g->stream));
        LAP_CUDA(g, cudaMemsetAsync(g->d_st_x2d, 0, nb, g->stream));
    }
    g->bpar_valid = false;
    g->st_omega = 0;
    g->st_cursor = 0;
    g->st_seed_set = false;
    g->ws_zeroed = false;                 // a failed earlier run may have left partial state
    g->pending = false;
    g->compact_disabled = false;
    g->fallbacks = 0;
    g->root = v;
    g->seed_set = false;
    g->omega = 0;
    g->cursor = 0;
    g->results_valid = false;
    g->err = "no error";
    if (root_out) *root_out = v;
    return LAP_OK;
}

lap_status lap_sample(lap_graph *g, uint64_t n_samples, uint64_t seed)
{
    return lap_sample_trace(g, n_samples, seed, nullptr, nullptr);
}

static lap_status sample_chunk(lap_graph *g, uint64_t n_samples, uint64_t seed, uint64_t *y1_dev, uint64_t *y2_dev,
                               double *m2_dev);

lap_status lap_sample_trace(lap_graph *g, uint64_t n_samples, uint64_t seed, uint64_t *y1_dev, uint64_t *y2_dev)
{
    if ((y1_dev == nullptr) != (y2_dev == nullptr)) return fail(g, LAP_ERR_INVALID_ARG, "y1_dev and y2_dev must both be set or both be NULL");
    // Launches of at most 2^24 samples bound the overflow list.
    const uint64_t chunk = 1ull << 24;
    for (uint64_t done = 0; done < n_samples || (n_samples == 0 && done == 0);) {
        const uint64_t c = n_samples - done < chunk ? n_samples - done : chunk;
        lap_status s = sample_chunk(g, c, seed, y1_dev ? y1_dev + done : nullptr, y2_dev ? y2_dev + done : nullptr,
                                    nullptr);
        if (s != LAP_OK || n_samples == 0) return s;
        done += c;
    }
    return LAP_OK;
}

lap_status lap_sample_trace_cv(lap_graph *g, uint64_t n_samples, uint64_t seed, uint64_t *y1_dev, uint64_t *y2_dev,
                               double *m2_dev)
{
    if (!g) return fail(nullptr, LAP_ERR_INVALID_ARG, "NULL handle");
    if (!y1_dev || !y2_dev || !m2_dev) return fail(g, LAP_ERR_INVALID_ARG, "y1_dev, y2_dev and m2_dev must be set");
    if (!g->cv2) return fail(g, LAP_ERR_INVALID_ARG, "the pi-walk potential (phi2) is not set");
    if (n_samples > (1ull << 24)) return fail(g, LAP_ERR_TOO_LARGE, "at most 2^24 samples per traced call");
    return sample_chunk(g, n_samples, seed, y1_dev, y2_dev, m2_dev);
}

static lap_status sample_chunk(lap_graph *g, uint64_t n_samples, uint64_t seed, uint64_t *y1_dev, uint64_t *y2_dev,
                               double *m2_dev)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    if (g->seed_set && seed != g->seed) return fail(g, LAP_ERR_INVALID_ARG, "seed differs from the seed in use since lap_set_root");
    if (g->cursor + n_samples > (1ull << 32)) return fail(g, LAP_ERR_TOO_LARGE, "sample ids are limited to 2^32");
    if (n_samples == 0) return LAP_OK;
    if ((s = resolve_pending(g)) != LAP_OK) return s;
    const int kernel = choose_kernel(g, n_samples);
    if ((s = ensure_workspace(g, kernel)) != LAP_OK) return s;
    g->seed = seed;
    g->seed_set = true;
    g->used_kernel = kernel;

    LapSampleLaunch p;
    memset(&p, 0, sizeof(p));
    p.g = LapDevGraph{g->d_rowinfo, g->d_col, g->n, g->arcs};
    p.root = g->root;
    p.seed = seed;
    p.first = (uint32_t)g->cursor;
    p.count = (uint32_t)n_samples;
    p.ws = g->ws;
    p.slot_epoch = g->d_slot_epoch;
    p.rep1 = g->d_rep1;
    p.cnt2 = g->d_cnt2;
    p.acc = g->d_acc;
    p.step_limit = g->step_limit ? g->step_limit : default_step_limit(g->n);
    p.block = g->block_opt;
    p.num_sms = g->num_sms;
    p.paths = g->paths_opt;
    p.ustart = g->path_start >= 0 ? (uint32_t)g->path_start + 1u : 0u;
    p.y1_out = reinterpret_cast<unsigned long long *>(y1_dev);
    p.y2_out = reinterpret_cast<unsigned long long *>(y2_dev);
    p.m2_out = m2_dev;
    if (g->cv1) {
        p.cv_h1 = g->d_cv_h1;
        p.cv_a1 = g->d_cv_a1;
    }
    if (g->cv2) {
        p.cv_h2 = g->d_cv_h2;
        p.cv_S2 = g->d_cv_S2;
        p.cv_a2 = g->d_cv_a2;
        p.cv_p2 = g->d_cv_p2;
    }
    if (kernel == LAP_KERNEL_COMPACT || kernel == LAP_KERNEL_GROUP) {
        if (g->ovf_cap < n_samples) {
            cudaFree(g->d_ovf_ids);
            g->d_ovf_ids = nullptr;
            g->ovf_cap = 0;
            if (dalloc(&g->d_ovf_ids, (size_t)n_samples) != cudaSuccess) {
                cudaGetLastError();
                return fail(g, LAP_ERR_OOM, "overflow list allocation failed");
            }
            g->ovf_cap = n_samples;
        }
        p.ovf_ids = g->d_ovf_ids;
    }
    if ((s = launch(g, p, kernel)) != LAP_OK) return s;
    if (kernel == LAP_KERNEL_COMPACT || kernel == LAP_KERNEL_GROUP) {
        g->pending = true;
        g->pending_launch = p;
    }
    g->omega += n_samples;
    g->cursor += n_samples;
    g->results_valid = false;
    return LAP_OK;
}

lap_status lap_sync(lap_graph *g)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    return poll_status(g);
}

static lap_status ensure_results(lap_graph *g)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    if (g->path_start >= 0)
        return fail(g, LAP_ERR_INVALID_ARG, "with a fixed walk start (LAP_OPT_PATH_START) the uniform-walk counts "
                                            "estimate a row of L_v^{-1}, not the ECC terms: use lap_lv_row");
    if (g->omega == 0) return fail(g, LAP_ERR_NO_SAMPLES, "no samples drawn");
    if ((s = poll_status(g)) != LAP_OK) return s;
    if (!g->results_valid) {
        LAP_CUDA(g, lap_launch_finalize(g->d_rowinfo, g->n, g->root, g->omega, g->d_rep1, g->d_cnt2,
                                        g->d_ldiag, g->d_ecc, g->d_red, g->stream));
        g->results_valid = true;
    }
    return LAP_OK;
}

static lap_status copy_out(lap_graph *g, void *out, const void *src, size_t bytes, int on_device)
{
    if (!out) return fail(g, LAP_ERR_INVALID_ARG, "output pointer is NULL");
    LAP_CUDA(g, cudaMemcpyAsync(out, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream));
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    return LAP_OK;
}

lap_status lap_ecc(lap_graph *g, double *out, int out_on_device)
{
    lap_status s = ensure_results(g);
    if (s != LAP_OK) return s;
    return copy_out(g, out, g->d_ecc, sizeof(double) * (size_t)g->n, out_on_device);
}

lap_status lap_ldiag(lap_graph *g, double *out, int out_on_device)
{
    lap_status s = ensure_results(g);
    if (s != LAP_OK) return s;
    return copy_out(g, out, g->d_ldiag, sizeof(double) * (size_t)g->n, out_on_device);
}

lap_status lap_kirchhoff(lap_graph *g, double *out1)
{
    lap_status s = ensure_results(g);
    if (s != LAP_OK) return s;
    return copy_out(g, out1, g->d_red + 1024 + 1, sizeof(double), 0);
}

lap_status lap_rw_betweenness(lap_graph *g, double *out, int out_on_device)
{
    lap_status s = ensure_results(g);
    if (s != LAP_OK) return s;
    if (!out) return fail(g, LAP_ERR_INVALID_ARG, "output pointer is NULL");
    double *dst = out;
    if (!out_on_device) {
        if (!g->d_aux && dalloc(&g->d_aux, (size_t)g->n) != cudaSuccess) {
            cudaGetLastError();
            return fail(g, LAP_ERR_OOM, "device allocation failed");
        }
        dst = g->d_aux;
    }
    LAP_CUDA(g, lap_launch_rw_betweenness(g->n, g->d_ldiag, g->d_red, dst, g->stream));
    if (out_on_device) {
        LAP_CUDA(g, cudaStreamSynchronize(g->stream));
        return LAP_OK;
    }
    return copy_out(g, out, g->d_aux, sizeof(double) * (size_t)g->n, 0);
}

lap_status lap_lv_row(lap_graph *g, double *out, int out_on_device)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (!out) return fail(g, LAP_ERR_INVALID_ARG, "output pointer is NULL");
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    if (g->omega == 0) return fail(g, LAP_ERR_NO_SAMPLES, "no samples drawn");
    if ((s = poll_status(g)) != LAP_OK) return s;
    if (out_on_device) {
        LAP_CUDA(g, lap_launch_lv_row(g->d_rowinfo, g->n, g->omega, g->d_cnt2, out, g->stream));
        LAP_CUDA(g, cudaStreamSynchronize(g->stream));
        return LAP_OK;
    }
    if (!g->d_aux && dalloc(&g->d_aux, (size_t)g->n) != cudaSuccess) {
        cudaGetLastError();
        return fail(g, LAP_ERR_OOM, "device allocation failed");
    }
    LAP_CUDA(g, lap_launch_lv_row(g->d_rowinfo, g->n, g->omega, g->d_cnt2, g->d_aux, g->stream));
    return copy_out(g, out, g->d_aux, sizeof(double) * (size_t)g->n, 0);
}

lap_status lap_lv_solve(lap_graph *g, const double *b, double *x, int on_device, double rtol, int32_t maxiter,
                        int32_t *iterations, double *residual)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (!b || !x) return fail(g, LAP_ERR_INVALID_ARG, "b and x must be set");
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    if (!(rtol > 0.0) || maxiter < 1) return fail(g, LAP_ERR_INVALID_ARG, "rtol must be > 0 and maxiter >= 1");
    const size_t n = (size_t)g->n;
    double *scratch = nullptr, *db = nullptr, *dx = nullptr;
    auto release = [&]() {
        cudaStreamSynchronize(g->stream);
        cudaFree(scratch);
        cudaFree(db);
        cudaFree(dx);
    };
    bool ok = dalloc(&scratch, 4 * n + 2 * 1024 + 8) == cudaSuccess;
    if (ok && !on_device) ok = dalloc(&db, n) == cudaSuccess && dalloc(&dx, n) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release();
        return fail(g, LAP_ERR_OOM, "solver scratch: device allocation failed");
    }
    cudaError_t e = cudaSuccess;
    if (!on_device) e = cudaMemcpyAsync(db, b, sizeof(double) * n, cudaMemcpyHostToDevice, g->stream);
    int32_t it = 0;
    double res = 0.0;
    if (e == cudaSuccess)
        e = lap_run_lv_solve(g->d_rowinfo, g->d_col, g->n, g->root, on_device ? b : db, on_device ? x : dx, scratch,
                             rtol, maxiter, &it, &res, g->stream);
    if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(x, dx, sizeof(double) * n, cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    release();
    if (e != cudaSuccess) return cuda_fail(g, e, "lap_lv_solve");
    if (iterations) *iterations = it;
    if (residual) *residual = res;
    return LAP_OK;
}

lap_status lap_kemeny(lap_graph *g, double *out1)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (!out1) return fail(g, LAP_ERR_INVALID_ARG, "output pointer is NULL");
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    if (g->omega == 0) return fail(g, LAP_ERR_NO_SAMPLES, "no samples drawn");
    if ((s = poll_status(g)) != LAP_OK) return s;
    LapDevAcc h;
    LAP_CUDA(g, cudaMemcpyAsync(&h, g->d_acc, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    // Alg. 4: kappa = (sum Y1 - sum Y2) / omega.
    *out1 = ((double)h.sum_y1 - (double)h.sum_y2) / (double)g->omega;
    return LAP_OK;
}

lap_status lap_counts(lap_graph *g, uint64_t *cnt1, uint64_t *cnt2, uint64_t *sums, int on_device)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    if ((s = poll_status(g)) != LAP_OK) return s;
    const size_t bytes = sizeof(uint64_t) * (size_t)g->n;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (cnt1) {
        // cnt1 = omega (the first visit of every non-root node) + repeats.
        LAP_CUDA(g, lap_launch_counts(g->n, g->root, g->omega, g->d_rep1,
                                      reinterpret_cast<unsigned long long *>(g->d_ldiag), g->stream));
        LAP_CUDA(g, cudaMemcpyAsync(cnt1, g->d_ldiag, bytes, kind, g->stream));
        g->results_valid = false;        // d_ldiag was used as scratch
    }
    if (cnt2) LAP_CUDA(g, cudaMemcpyAsync(cnt2, g->d_cnt2, bytes, kind, g->stream));
    if (sums) {
        LapDevAcc h;
        LAP_CUDA(g, cudaMemcpyAsync(&h, g->d_acc, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
        LAP_CUDA(g, cudaStreamSynchronize(g->stream));
        uint64_t v4[4] = {g->omega, h.sum_y1, h.sum_y2, g->seed};
        if (on_device) LAP_CUDA(g, cudaMemcpyAsync(sums, v4, sizeof(v4), cudaMemcpyHostToDevice, g->stream));
        else memcpy(sums, v4, sizeof(v4));
    }
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    return LAP_OK;
}

lap_status lap_set_counts(lap_graph *g, const uint64_t *cnt1, const uint64_t *cnt2, const uint64_t *sums, int on_device)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    if (!cnt1 || !cnt2 || !sums) return fail(g, LAP_ERR_INVALID_ARG, "cnt1, cnt2 and sums must be set");
    if ((s = poll_status(g)) != LAP_OK) return s;
    uint64_t h3[3];
    const size_t bytes = sizeof(uint64_t) * (size_t)g->n;
    if (on_device) {
        LAP_CUDA(g, cudaMemcpyAsync(h3, sums, sizeof(h3), cudaMemcpyDeviceToHost, g->stream));
        LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    } else {
        memcpy(h3, sums, sizeof(h3));
    }
    if (h3[0] == 0) return fail(g, LAP_ERR_INVALID_ARG, "omega (sums[0]) must be >= 1");
    // cnt1 is staged in the ldiag buffer (finalize overwrites it anyway).
    unsigned long long *stage = reinterpret_cast<unsigned long long *>(g->d_ldiag);
    unsigned int *bad = reinterpret_cast<unsigned int *>(g->d_red);
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    LAP_CUDA(g, cudaMemcpyAsync(stage, cnt1, bytes, kind, g->stream));
    LAP_CUDA(g, cudaMemsetAsync(bad, 0, sizeof(unsigned int), g->stream));
    LAP_CUDA(g, lap_launch_rep_from_counts(g->n, g->root, h3[0], stage, g->d_rep1, bad, g->stream));
    unsigned int hb = 0;
    LAP_CUDA(g, cudaMemcpyAsync(&hb, bad, sizeof(hb), cudaMemcpyDeviceToHost, g->stream));
    LAP_CUDA(g, cudaMemcpyAsync(g->d_cnt2, cnt2, bytes, kind, g->stream));
    LapDevAcc acc;
    memset(&acc, 0, sizeof(acc));
    acc.sum_y1 = h3[1];
    acc.sum_y2 = h3[2];
    LAP_CUDA(g, cudaMemcpyAsync(g->d_acc, &acc, sizeof(acc), cudaMemcpyHostToDevice, g->stream));
    if (g->d_cv_a1) {
        LAP_CUDA(g, cudaMemsetAsync(g->d_cv_a1, 0, bytes, g->stream));
        LAP_CUDA(g, cudaMemsetAsync(g->d_cv_a2, 0, bytes, g->stream));
        LAP_CUDA(g, cudaMemsetAsync(g->d_cv_p2, 0, bytes, g->stream));
    }
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    g->omega = h3[0];
    g->results_valid = false;
    if (hb) {
        LAP_CUDA(g, cudaMemsetAsync(g->d_rep1, 0, bytes, g->stream));
        LAP_CUDA(g, cudaMemsetAsync(g->d_cnt2, 0, bytes, g->stream));
        LAP_CUDA(g, cudaMemsetAsync(g->d_acc, 0, sizeof(LapDevAcc), g->stream));
        LAP_CUDA(g, cudaStreamSynchronize(g->stream));
        g->omega = 0;
        return fail(g, LAP_ERR_INVALID_ARG, "counts inconsistent with omega samples (cnt1[v] != 0 or cnt1[u] < omega)");
    }
    return LAP_OK;
}

// ------------------------------------------------------------ SpanTree (Alg. 1, Alg. 3)

static lap_status spantree_prepare(lap_graph *g)
{
    const size_t n = (size_t)g->n;
    if (!g->d_st_x1) {
        bool ok = dalloc(&g->d_st_x1, n) == cudaSuccess && dalloc(&g->d_st_x2, n) == cudaSuccess &&
                  dalloc(&g->d_st_x2d, n) == cudaSuccess && dalloc(&g->d_st_rep1, n) == cudaSuccess &&
                  dalloc(&g->d_st_ldiag, n) == cudaSuccess && dalloc(&g->d_st_ecc, n) == cudaSuccess &&
                  dalloc(&g->d_st_red, 1024 + 8) == cudaSuccess && dalloc(&g->d_st_acc, 1) == cudaSuccess &&
                  dalloc(&g->d_bpar, n) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return fail(g, LAP_ERR_OOM, "SpanTree allocation failed");
        }
        const size_t nb = sizeof(unsigned long long) * n;
        LAP_CUDA(g, cudaMemsetAsync(g->d_st_x1, 0, nb, g->stream));
        LAP_CUDA(g, cudaMemsetAsync(g->d_st_x2, 0, nb, g->stream));
        LAP_CUDA(g, cudaMemsetAsync(g->d_st_x2d, 0, nb, g->stream));
        g->bpar_valid = false;
    }
    if (!g->bpar_valid) {
        LAP_CUDA(g, cudaMemsetAsync(g->d_st_acc, 0, sizeof(LapDevAcc), g->stream));
        LAP_CUDA(g, lap_launch_bfs_parent(g->d_rowinfo, g->d_col, g->d_hops, g->n, g->root, g->d_bpar,
                                          &g->d_st_acc->status, g->stream));
        g->bpar_valid = true;
    }
    if (!g->d_st_scratch) {
        // One scratch region per tree CTA: two CTAs per SM, fewer if memory is short.
        const uint64_t per = lap_spantree_scratch_ints(g->n) * sizeof(int32_t);
        for (int b = 2 * g->num_sms; b >= 1; b /= 2) {
            if (cudaMalloc(&g->d_st_scratch, per * (uint64_t)b) == cudaSuccess) {
                g->st_blocks = b;
                break;
            }
            cudaGetLastError();
            g->d_st_scratch = nullptr;
        }
        if (!g->d_st_scratch) return fail(g, LAP_ERR_OOM, "SpanTree scratch allocation failed");
    }
    return LAP_OK;
}

lap_status lap_spantree_sample(lap_graph *g, uint64_t n_samples, uint64_t seed)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    if (g->st_seed_set && seed != g->st_seed) return fail(g, LAP_ERR_INVALID_ARG, "seed differs from the SpanTree seed in use since lap_set_root");
    if (g->st_cursor + n_samples > (1ull << 32)) return fail(g, LAP_ERR_TOO_LARGE, "sample ids are limited to 2^32");
    if (n_samples == 0) return LAP_OK;
    if ((s = resolve_pending(g)) != LAP_OK) return s;      // the workspace is about to be reused
    if ((s = spantree_prepare(g)) != LAP_OK) return s;
    if ((s = ensure_workspace(g, LAP_KERNEL_WIDE)) != LAP_OK) return s;
    g->st_seed = seed;
    g->st_seed_set = true;
    const uint64_t per_tree = 8ull * (uint64_t)g->n;
    uint64_t cap = g->ws_bytes / per_tree;
    if (cap > g->slot_epoch_cap) cap = g->slot_epoch_cap;
    if (cap > (1ull << 24)) cap = 1ull << 24;
    if (cap == 0) return fail(g, LAP_ERR_OOM, "workspace smaller than one tree");
    const uint64_t limit = g->step_limit ? g->step_limit : default_step_limit(g->n);
    for (uint64_t done = 0; done < n_samples;) {
        const uint64_t c = n_samples - done < cap ? n_samples - done : cap;
        LapSampleLaunch p;
        memset(&p, 0, sizeof(p));
        p.g = LapDevGraph{g->d_rowinfo, g->d_col, g->n, g->arcs};
        p.root = g->root;
        p.seed = seed;
        p.first = (uint32_t)(g->st_cursor + done);
        p.count = (uint32_t)c;
        p.slots = c;
        p.ws = g->ws;
        p.slot_epoch = g->d_slot_epoch;
        p.rep1 = g->d_st_rep1;
        p.cnt2 = g->d_st_rep1;
        p.acc = g->d_st_acc;
        p.step_limit = limit;
        p.block = g->block_opt;
        p.num_sms = g->num_sms;
        p.flags = LAP_SAMPLE_ONE_PER_LANE | LAP_SAMPLE_WILSON_ONLY;
        LAP_CUDA(g, lap_launch_sample(p, g->stream));
        LapSpanTreeLaunch t;
        memset(&t, 0, sizeof(t));
        t.rowinfo = g->d_rowinfo;
        t.bpar = g->d_bpar;
        t.trees = reinterpret_cast<const unsigned long long *>(g->ws);
        t.n = g->n;
        t.root = g->root;
        t.count = (uint32_t)c;
        t.scratch = g->d_st_scratch;
        t.scratch_ints = lap_spantree_scratch_ints(g->n);
        t.x1 = g->d_st_x1;
        t.x2 = g->d_st_x2;
        t.x2d = g->d_st_x2d;
        t.status = &g->d_st_acc->status;
        LAP_CUDA(g, lap_launch_spantree(t, (int)(c < (uint64_t)g->st_blocks ? c : (uint64_t)g->st_blocks), g->stream));
        done += c;
    }
    LapDevAcc h;
    LAP_CUDA(g, cudaMemcpyAsync(&h, g->d_st_acc, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    if (h.status & LAP_DEV_STEP_LIMIT) {
        g->sticky = LAP_ERR_STEP_LIMIT;
        return fail(g, LAP_ERR_STEP_LIMIT, "a Wilson run exceeded the per-sample step budget (LAP_OPT_STEP_LIMIT)");
    }
    if (h.status) {
        g->sticky = LAP_ERR_CUDA;
        return fail(g, LAP_ERR_CUDA, "internal error in the SpanTree kernels (status " + std::to_string(h.status) + ")");
    }
    g->st_cursor += n_samples;
    g->st_omega += n_samples;
    return LAP_OK;
}

lap_status lap_spantree_sums(lap_graph *g, int64_t *x1, int64_t *x2, int64_t *x2d, uint64_t *omega, int on_device)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    if (omega) *omega = g->st_omega;
    if (!g->d_st_x1) {
        if (x1 || x2 || x2d) return fail(g, LAP_ERR_NO_SAMPLES, "no SpanTree samples drawn");
        return LAP_OK;
    }
    const size_t nb = sizeof(int64_t) * (size_t)g->n;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (x1) LAP_CUDA(g, cudaMemcpyAsync(x1, g->d_st_x1, nb, kind, g->stream));
    if (x2) LAP_CUDA(g, cudaMemcpyAsync(x2, g->d_st_x2, nb, kind, g->stream));
    if (x2d) LAP_CUDA(g, cudaMemcpyAsync(x2d, g->d_st_x2d, nb, kind, g->stream));
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    return LAP_OK;
}

lap_status lap_spantree_estimates(lap_graph *g, double *ldiag, double *ecc, int on_device, double *kemeny)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    if (g->st_omega == 0) return fail(g, LAP_ERR_NO_SAMPLES, "no SpanTree samples drawn");
    LAP_CUDA(g, lap_launch_spantree_finalize(g->d_rowinfo, g->n, g->root, g->st_omega,
                                             reinterpret_cast<const long long *>(g->d_st_x1),
                                             reinterpret_cast<const long long *>(g->d_st_x2),
                                             reinterpret_cast<const long long *>(g->d_st_x2d), g->d_st_ldiag,
                                             g->d_st_ecc, g->d_st_red, g->stream));
    const size_t nb = sizeof(double) * (size_t)g->n;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (ldiag) LAP_CUDA(g, cudaMemcpyAsync(ldiag, g->d_st_ldiag, nb, kind, g->stream));
    if (ecc) LAP_CUDA(g, cudaMemcpyAsync(ecc, g->d_st_ecc, nb, kind, g->stream));
    double sums[2] = {0.0, 0.0};
    LAP_CUDA(g, cudaMemcpyAsync(sums, g->d_st_red + 1024 + 2, sizeof(sums), cudaMemcpyDeviceToHost, g->stream));
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    // Alg. 3: kappa = (sum_u d_u X1[u]) / omega - (sum_u d_u X2d[u]) / (2m omega).
    const double w = (double)g->st_omega;
    if (kemeny) *kemeny = sums[0] / w - sums[1] / ((double)g->arcs * w);
    return LAP_OK;
}

lap_status lap_hops(lap_graph *g, int32_t *out, int on_device)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    return copy_out(g, out, g->d_hops, sizeof(int32_t) * (size_t)g->n, on_device);
}

lap_status lap_features(lap_graph *g, float *feat_dev)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (!feat_dev) return fail(g, LAP_ERR_INVALID_ARG, "feat_dev is NULL");
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    if (!g->d_feat_scratch && dalloc(&g->d_feat_scratch, 5 * (size_t)g->n) != cudaSuccess) {
        cudaGetLastError();
        return fail(g, LAP_ERR_OOM, "feature scratch allocation failed");
    }
    LAP_CUDA(g, lap_launch_features(g->d_rowinfo, g->d_col, g->d_hops, g->n, g->root, g->d_feat_scratch, feat_dev,
                                    g->stream));
    return LAP_OK;
}

lap_status lap_hitting_walks(lap_graph *g, uint32_t reps, uint64_t seed, uint64_t *sums_dev)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (!sums_dev || reps == 0) return fail(g, LAP_ERR_INVALID_ARG, "sums_dev must be set and reps >= 1");
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    if ((s = resolve_pending(g)) != LAP_OK) return s;
    LAP_CUDA(g, cudaMemsetAsync(sums_dev, 0, sizeof(uint64_t) * (size_t)g->n, g->stream));
    unsigned int *status = reinterpret_cast<unsigned int *>(g->d_red);
    LAP_CUDA(g, cudaMemsetAsync(status, 0, sizeof(unsigned int), g->stream));
    const uint64_t limit = g->step_limit ? g->step_limit : default_step_limit(g->n);
    LAP_CUDA(g, lap_launch_hitting_walks(LapDevGraph{g->d_rowinfo, g->d_col, g->n, g->arcs}, g->root, seed, reps, limit,
                                         reinterpret_cast<unsigned long long *>(sums_dev), status, g->num_sms,
                                         g->stream));
    unsigned int h = 0;
    LAP_CUDA(g, cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    if (h & LAP_DEV_STEP_LIMIT) return fail(g, LAP_ERR_STEP_LIMIT, "a hitting walk exceeded the step budget");
    return LAP_OK;
}

lap_status lap_cv_targets(lap_graph *g, uint32_t reps, uint64_t seed, float *targets_dev)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (!targets_dev || reps == 0) return fail(g, LAP_ERR_INVALID_ARG, "targets_dev must be set and reps >= 1");
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    if (g->omega == 0) return fail(g, LAP_ERR_NO_SAMPLES, "no samples drawn");
    if ((s = poll_status(g)) != LAP_OK) return s;
    if (!g->d_aux && dalloc(&g->d_aux, (size_t)g->n) != cudaSuccess) {
        cudaGetLastError();
        return fail(g, LAP_ERR_OOM, "device allocation failed");
    }
    uint64_t *hit = reinterpret_cast<uint64_t *>(g->d_aux);
    if ((s = lap_hitting_walks(g, reps, seed, hit)) != LAP_OK) return s;
    LapDevAcc h;
    LAP_CUDA(g, cudaMemcpyAsync(&h, g->d_acc, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    // E[Y2] estimated from the samples drawn; kept away from 0 for graphs
    // whose pi-walks all start at the root.
    double mean_y2 = (double)h.sum_y2 / (double)g->omega;
    if (!(mean_y2 > 1e-9)) mean_y2 = 1e-9;
    LAP_CUDA(g, lap_launch_cv_targets(g->n, g->root, g->omega, g->d_rep1,
                                      reinterpret_cast<const unsigned long long *>(hit), reps, mean_y2, targets_dev,
                                      g->stream));
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    return LAP_OK;
}

lap_status lap_cv_potentials(lap_graph *g, const float *y_dev, double *phi1_dev, double *phi2_dev)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (!y_dev || (!phi1_dev && !phi2_dev)) return fail(g, LAP_ERR_INVALID_ARG, "y_dev and one output must be set");
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    double scale2 = 0.0;
    if (phi2_dev) {
        if (g->omega == 0) return fail(g, LAP_ERR_NO_SAMPLES, "phi2 is scaled by the mean Y2 of the samples drawn: none drawn");
        if ((s = poll_status(g)) != LAP_OK) return s;
        LapDevAcc h;
        LAP_CUDA(g, cudaMemcpyAsync(&h, g->d_acc, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
        LAP_CUDA(g, cudaStreamSynchronize(g->stream));
        scale2 = (double)h.sum_y2 / (double)g->omega;
    }
    LAP_CUDA(g, lap_launch_cv_potentials(g->d_rowinfo, g->n, g->root, y_dev, scale2, phi1_dev, phi2_dev, g->stream));
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    return LAP_OK;
}

lap_status lap_cv_fit_betas(lap_graph *g, const double *phi1_dev, const double *phi2_dev, uint64_t seed,
                            uint64_t first_id, uint64_t pilot, uint32_t batches, double *beta1, double *beta2)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (!beta1 || !beta2 || (!phi1_dev && !phi2_dev)) return fail(g, LAP_ERR_INVALID_ARG, "beta outputs and one potential must be set");
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    if (g->omega != 0) return fail(g, LAP_ERR_INVALID_ARG, "the pilot batches must be the first samples after lap_set_root");
    if (batches < 2 || batches > 64) return fail(g, LAP_ERR_INVALID_ARG, "batches must be in [2, 64]");
    const uint64_t per = pilot / batches;
    if (per < 1 || per > (1ull << 24)) return fail(g, LAP_ERR_INVALID_ARG, "pilot / batches must be in [1, 2^24]");
    const uint64_t total = per * batches;
    if (first_id >= (1ull << 32) || total > (1ull << 32) - first_id)
        return fail(g, LAP_ERR_TOO_LARGE, "pilot sample ids must lie below 2^32");
    const int32_t root = g->root;
    const size_t n = (size_t)g->n;
    if ((s = lap_cv_set_potentials(g, phi1_dev, phi2_dev)) != LAP_OK) return s;
    g->cursor = first_id;

    double *vb = nullptr, *zb = nullptr, *m2 = nullptr, *red = nullptr;
    long long *prev = nullptr;
    unsigned long long *y1 = nullptr, *y2 = nullptr;
    auto release = [&]() {
        cudaStreamSynchronize(g->stream);
        cudaFree(vb); cudaFree(zb); cudaFree(m2); cudaFree(red); cudaFree(prev); cudaFree(y1); cudaFree(y2);
    };
    bool ok = dalloc(&y1, (size_t)total) == cudaSuccess && dalloc(&y2, (size_t)total) == cudaSuccess &&
              dalloc(&red, 2 * 1024 + 8) == cudaSuccess;
    if (ok && phi2_dev) ok = dalloc(&m2, (size_t)total) == cudaSuccess;
    if (ok && phi1_dev)
        ok = dalloc(&vb, n * batches) == cudaSuccess && dalloc(&zb, n * batches) == cudaSuccess &&
             dalloc(&prev, 2 * n) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        release();
        return fail(g, LAP_ERR_OOM, "pilot buffers: device allocation failed");
    }
    if (cudaMemsetAsync(red, 0, sizeof(double) * (2 * 1024 + 8), g->stream) != cudaSuccess ||
        (prev && cudaMemsetAsync(prev, 0, sizeof(long long) * 2 * n, g->stream) != cudaSuccess)) {
        release();
        return fail(g, LAP_ERR_CUDA, "cudaMemsetAsync failed");
    }
    for (uint32_t b = 0; b < batches && s == LAP_OK; ++b) {
        s = sample_chunk(g, per, seed, reinterpret_cast<uint64_t *>(y1 + b * per),
                         reinterpret_cast<uint64_t *>(y2 + b * per), m2 ? m2 + b * per : nullptr);
        if (s == LAP_OK) s = resolve_pending(g);      // re-runs of withdrawn samples complete the batch
        if (s == LAP_OK && phi1_dev) {
            const cudaError_t e = lap_launch_beta1_batch(g->d_rowinfo, g->n, root, g->omega, g->d_rep1,
                                                         reinterpret_cast<const long long *>(g->d_cv_a1), g->d_cv_S1,
                                                         prev, prev + n, vb + b * n, zb + b * n, g->stream);
            if (e != cudaSuccess) s = cuda_fail(g, e, "beta1 batch");
        }
    }
    if (s == LAP_OK) s = poll_status(g);
    double out[4] = {0.0, 0.0, 0.0, 0.0};
    if (s == LAP_OK) {
        cudaError_t e = cudaSuccess;
        if (phi1_dev) e = lap_launch_beta1_reduce(g->n, (int32_t)batches, vb, zb, red, red + 2 * 1024 + 2, g->stream);
        if (e == cudaSuccess && phi2_dev) e = lap_launch_beta2_reduce(y1, y2, m2, (int64_t)total, red, red + 2 * 1024 + 4, g->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, red + 2 * 1024 + 2, sizeof(out), cudaMemcpyDeviceToHost, g->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) s = cuda_fail(g, e, "beta reductions");
    }
    release();
    if (s != LAP_OK) return s;
    // Least squares: beta1 = cov(V, Z1/d) / var(Z1/d) pooled over nodes;
    // beta2 = -cov(Y1 - Y2, M2) / var(M2) (the Kemeny CV adds + beta2 M2).
    *beta1 = out[1] > 0.0 ? out[0] / out[1] : 0.0;
    *beta2 = out[3] > 0.0 ? -out[2] / out[3] : 0.0;
    // Back to the state after lap_set_root, the potentials kept: the pilot
    // samples are not part of any estimate.
    return lap_set_root(g, root, nullptr);
}

lap_status lap_cv_set_potentials(lap_graph *g, const double *phi1_dev, const double *phi2_dev)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (g->omega != 0) return fail(g, LAP_ERR_INVALID_ARG, "potentials can only be set before the first sample after lap_set_root");
    const size_t n = (size_t)g->n;
    if ((phi1_dev || phi2_dev) && !g->d_cv_a1) {
        bool ok = dalloc(&g->d_cv_h1, n) == cudaSuccess && dalloc(&g->d_cv_S1, n) == cudaSuccess &&
                  dalloc(&g->d_cv_h2, n) == cudaSuccess && dalloc(&g->d_cv_S2, n) == cudaSuccess &&
                  dalloc(&g->d_cv_a1, n) == cudaSuccess && dalloc(&g->d_cv_a2, n) == cudaSuccess &&
                  dalloc(&g->d_cv_p2, n) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            return fail(g, LAP_ERR_OOM, "control-variate allocation failed");
        }
        const size_t nb = sizeof(unsigned long long) * n;
        LAP_CUDA(g, cudaMemsetAsync(g->d_cv_a1, 0, nb, g->stream));
        LAP_CUDA(g, cudaMemsetAsync(g->d_cv_a2, 0, nb, g->stream));
        LAP_CUDA(g, cudaMemsetAsync(g->d_cv_p2, 0, nb, g->stream));
    }
    g->cv1 = phi1_dev != nullptr;
    g->cv2 = phi2_dev != nullptr;
    if (phi1_dev) LAP_CUDA(g, lap_launch_potential(g->d_rowinfo, g->d_col, g->n, phi1_dev, g->d_cv_h1, g->d_cv_S1, g->stream));
    if (phi2_dev) LAP_CUDA(g, lap_launch_potential(g->d_rowinfo, g->d_col, g->n, phi2_dev, g->d_cv_h2, g->d_cv_S2, g->stream));
    g->results_valid = false;
    return LAP_OK;
}

lap_status lap_cv_sums(lap_graph *g, int64_t *a1, int64_t *a2, int64_t *p2, int on_device)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (!g->d_cv_a1) return fail(g, LAP_ERR_INVALID_ARG, "no potentials set");
    if ((s = poll_status(g)) != LAP_OK) return s;
    const size_t nb = sizeof(int64_t) * (size_t)g->n;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (a1) LAP_CUDA(g, cudaMemcpyAsync(a1, g->d_cv_a1, nb, kind, g->stream));
    if (a2) LAP_CUDA(g, cudaMemcpyAsync(a2, g->d_cv_a2, nb, kind, g->stream));
    if (p2) LAP_CUDA(g, cudaMemcpyAsync(p2, g->d_cv_p2, nb, kind, g->stream));
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    return LAP_OK;
}

lap_status lap_cv_set_sums(lap_graph *g, const int64_t *a1, const int64_t *a2, const int64_t *p2, int on_device)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (!g->d_cv_a1) return fail(g, LAP_ERR_INVALID_ARG, "no potentials set");
    if (!a1 || !a2 || !p2) return fail(g, LAP_ERR_INVALID_ARG, "a1, a2 and p2 must be set");
    if ((s = poll_status(g)) != LAP_OK) return s;
    const size_t nb = sizeof(int64_t) * (size_t)g->n;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    LAP_CUDA(g, cudaMemcpyAsync(g->d_cv_a1, a1, nb, kind, g->stream));
    LAP_CUDA(g, cudaMemcpyAsync(g->d_cv_a2, a2, nb, kind, g->stream));
    LAP_CUDA(g, cudaMemcpyAsync(g->d_cv_p2, p2, nb, kind, g->stream));
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    g->results_valid = false;
    return LAP_OK;
}

lap_status lap_cv_estimates(lap_graph *g, double beta1, double beta2, double *ldiag, double *ecc, int on_device,
                            double *kemeny, double *m2_total)
{
    lap_status s = check_sticky(g);
    if (s != LAP_OK) return s;
    if (g->root < 0) return fail(g, LAP_ERR_NO_ROOT, "lap_set_root has not been called");
    if (g->omega == 0) return fail(g, LAP_ERR_NO_SAMPLES, "no samples drawn");
    if (g->path_start >= 0 && (ldiag || ecc))
        return fail(g, LAP_ERR_INVALID_ARG, "with a fixed walk start (LAP_OPT_PATH_START) there are no ECC estimates");
    if ((s = poll_status(g)) != LAP_OK) return s;
    double *m2d = g->d_red + 1024 + 4;
    LAP_CUDA(g, cudaMemsetAsync(m2d, 0, sizeof(double), g->stream));
    LAP_CUDA(g, lap_launch_cv_finalize(g->d_rowinfo, g->n, g->root, g->omega, g->d_rep1, g->d_cnt2,
                                       g->cv1 ? reinterpret_cast<const long long *>(g->d_cv_a1) : nullptr, g->d_cv_S1, beta1,
                                       g->cv2 ? reinterpret_cast<const long long *>(g->d_cv_a2) : nullptr,
                                       reinterpret_cast<const long long *>(g->d_cv_p2), g->d_cv_S2,
                                       g->d_ldiag, g->d_ecc, g->d_red, m2d, g->stream));
    g->results_valid = false;          // the plain results were overwritten
    const size_t nb = sizeof(double) * (size_t)g->n;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (ldiag) LAP_CUDA(g, cudaMemcpyAsync(ldiag, g->d_ldiag, nb, kind, g->stream));
    if (ecc) LAP_CUDA(g, cudaMemcpyAsync(ecc, g->d_ecc, nb, kind, g->stream));
    double m2 = 0.0;
    LAP_CUDA(g, cudaMemcpyAsync(&m2, m2d, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    LapDevAcc h;
    LAP_CUDA(g, cudaMemcpyAsync(&h, g->d_acc, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
    LAP_CUDA(g, cudaStreamSynchronize(g->stream));
    if (m2_total) *m2_total = m2;
    // Alg. 4 with the control variate: kappa = (sum Y1 - sum Y2 + beta2 M2) / omega.
    if (kemeny) *kemeny = (((double)h.sum_y1 - (double)h.sum_y2) + beta2 * m2) / (double)g->omega;
    return LAP_OK;
}

lap_status lap_mlp_select(int32_t kernel)
{
    if (kernel != LAP_MLP_TCGEN05 && kernel != LAP_MLP_MMA_SYNC)
        return fail(nullptr, LAP_ERR_INVALID_ARG, "MLP kernel must be LAP_MLP_TCGEN05 or LAP_MLP_MMA_SYNC");
    g_mlp_kernel.store(kernel);
    return LAP_OK;
}

lap_status lap_mlp_forward(const float *params_dev, const float *x_dev, int64_t rows, float *y_dev, void *cuda_stream)
{
    if (!params_dev || !x_dev || !y_dev || rows < 0) return fail(nullptr, LAP_ERR_INVALID_ARG, "bad MLP arguments");
    cudaError_t e = launch_mlp(params_dev, x_dev, nullptr, rows, 0.f, 0.f, y_dev, nullptr, nullptr,
                               reinterpret_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? LAP_OK : cuda_fail(nullptr, e, "lap_mlp_forward");
}

lap_status lap_mlp_loss_grad(const float *params_dev, const float *x_dev, const float *t_dev, int64_t rows, float w0,
                             float w1, float *grad_dev, float *loss_dev, void *cuda_stream)
{
    if (!params_dev || !x_dev || !t_dev || !grad_dev || !loss_dev || rows <= 0)
        return fail(nullptr, LAP_ERR_INVALID_ARG, "bad MLP arguments");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMemsetAsync(grad_dev, 0, sizeof(float) * LAP_MLP_PARAMS, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(loss_dev, 0, sizeof(float), st);
    if (e == cudaSuccess) e = launch_mlp(params_dev, x_dev, t_dev, rows, w0, w1, nullptr, grad_dev, loss_dev, st);
    return e == cudaSuccess ? LAP_OK : cuda_fail(nullptr, e, "lap_mlp_loss_grad");
}

lap_status lap_adamw(float *params_dev, float *m_dev, float *v_dev, const float *grad_dev, int64_t count, int32_t step,
                     float lr, float beta1, float beta2, float eps, float weight_decay, void *cuda_stream)
{
    if (!params_dev || !m_dev || !v_dev || !grad_dev || count <= 0 || step < 1)
        return fail(nullptr, LAP_ERR_INVALID_ARG, "bad AdamW arguments");
    cudaError_t e = lap_launch_adamw(params_dev, m_dev, v_dev, grad_dev, count, step, lr, beta1, beta2, eps, weight_decay,
                                     reinterpret_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? LAP_OK : cuda_fail(nullptr, e, "lap_adamw");
}

lap_status lap_graph_info(const lap_graph *g, int32_t *n, int64_t *arcs, int32_t *root)
{
    if (!g) return fail(nullptr, LAP_ERR_INVALID_ARG, "NULL handle");
    if (n) *n = g->n;
    if (arcs) *arcs = g->arcs;
    if (root) *root = g->root;
    return LAP_OK;
}

}  // extern "C"
