// lap_sample_static: the LEWalk sampler for callers that cannot allocate
// device memory (see include/lap.h).  All scratch the sampler needs lives in
// one file-scope device array, so the call performs no cudaMalloc/cudaFree
// and uses no allocating library routine.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "lap_internal.h"

namespace {

// Fixed scratch: per-node row records, per-node repeat-visit counters, the
// device accumulators, per-slot epoch bits and the 8-byte-per-node Wilson
// state of as many sample slots as fit.  Every GPU that loads this library holds it until the process exits.
constexpr uint64_t kStaticScratchBytes = 32ull << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};
void *g_scratch_ctx[kMaxDevices] = {};

// The driver's cuCtxGetCurrent, fetched through the runtime so that the
// library keeps no link-time dependency on the driver library.
typedef int (*CtxGetCurrentFn)(void **);

void *current_context()
{
    static CtxGetCurrentFn fn = [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(f);
    }();
    void *ctx = nullptr;
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}

uint64_t round256(uint64_t x) { return (x + 255ull) & ~255ull; }

// Device address of g_static_scratch on the current device.  The host-side
// symbol is only a stand-in, so the address is looked up once per device
// with that device current.  The lookup is repeated when the device's
// context has changed since (after a cudaDeviceReset the runtime creates a
// new context, in which the array has a new address).
lap_status scratch_address(void **out, std::string &err)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { err = std::string("cudaGetDevice: ") + cudaGetErrorString(e); return LAP_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) { err = "device index out of range"; return LAP_ERR_INVALID_ARG; }
    // The current context (NULL before this thread's first runtime call, or
    // before the runtime has initialised the driver).
    void *ctx = current_context();
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev] || !ctx || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return LAP_ERR_CUDA;
        }
        ctx = current_context();
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return LAP_OK;
}

thread_local std::string g_static_error = "no error";

lap_status fail_static(lap_status s, const std::string &m)
{
    g_static_error = m;
    return s;
}

#define STATIC_CUDA(call)                                                                     \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail_static(LAP_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

}  // namespace

extern "C" {

const char *lap_static_last_error(void) { return g_static_error.c_str(); }

uint64_t lap_static_scratch_bytes(void) { return kStaticScratchBytes; }

lap_status lap_sample_static(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t root,
                             uint64_t seed, uint64_t first_id, uint64_t n_samples,
                             uint64_t *cnt1, uint64_t *cnt2, uint64_t *sums2, void *cuda_stream)
{
    if (n < 2 || !row_ptr || !col_idx || !cnt1 || !cnt2 || !sums2)
        return fail_static(LAP_ERR_INVALID_ARG, "n must be >= 2 and every pointer set");
    if (root >= n) return fail_static(LAP_ERR_INVALID_ARG, "root out of range");
    if (n_samples == 0) return fail_static(LAP_ERR_INVALID_ARG, "n_samples must be >= 1");
    // Ids are 32-bit: [first_id, first_id + n_samples) must lie in [0, 2^32)
    // (written so that no sum can wrap).
    if (first_id >= (1ull << 32) || n_samples > (1ull << 32) - first_id)
        return fail_static(LAP_ERR_TOO_LARGE, "sample ids [first_id, first_id + n_samples) must lie below 2^32");

    // Layout of the static scratch.
    const uint64_t rowinfo_bytes = round256(8ull * (uint64_t)n);
    const uint64_t rep_bytes = round256(8ull * (uint64_t)n);
    const uint64_t acc_bytes = round256(sizeof(LapDevAcc));
    const uint64_t state_per_slot = 8ull * (uint64_t)n;
    const uint64_t fixed = rowinfo_bytes + rep_bytes + acc_bytes;
    if (fixed + round256(4) + state_per_slot > kStaticScratchBytes) {
        char buf[200];
        snprintf(buf, sizeof(buf), "graph too large for the %llu-byte static scratch: n = %d needs %llu bytes for one sample",
                 (unsigned long long)kStaticScratchBytes, n, (unsigned long long)(fixed + 256 + state_per_slot));
        return fail_static(LAP_ERR_TOO_LARGE, buf);
    }
    uint64_t slots = (kStaticScratchBytes - fixed - 256) / (state_per_slot + 4);
    while (slots > 1 && fixed + round256(4 * slots) + slots * state_per_slot > kStaticScratchBytes) --slots;
    if (slots > n_samples) slots = n_samples;

    void *base = nullptr;
    std::string err;
    lap_status s = scratch_address(&base, err);
    if (s != LAP_OK) return fail_static(s, err);
    unsigned char *b = static_cast<unsigned char *>(base);
    int2 *rowinfo = reinterpret_cast<int2 *>(b);
    unsigned long long *rep = reinterpret_cast<unsigned long long *>(b + rowinfo_bytes);
    LapDevAcc *acc = reinterpret_cast<LapDevAcc *>(b + rowinfo_bytes + rep_bytes);
    unsigned int *slot_epoch = reinterpret_cast<unsigned int *>(b + fixed);
    void *state = b + fixed + round256(4 * slots);

    int dev = 0, num_sms = 1;
    STATIC_CUDA(cudaGetDevice(&dev));
    STATIC_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);

    // The array keeps the previous call's contents: clear everything that
    // must start at zero (counters, accumulators, epochs, Wilson state).
    STATIC_CUDA(cudaMemsetAsync(rep, 0, 8ull * (uint64_t)n, st));
    STATIC_CUDA(cudaMemsetAsync(acc, 0, sizeof(LapDevAcc), st));
    STATIC_CUDA(cudaMemsetAsync(slot_epoch, 0, 4 * slots, st));
    STATIC_CUDA(cudaMemsetAsync(state, 0, slots * state_per_slot, st));
    STATIC_CUDA(cudaMemsetAsync(cnt2, 0, sizeof(uint64_t) * (size_t)n, st));
    STATIC_CUDA(lap_launch_rowinfo(row_ptr, n, rowinfo, st));

    if (root < 0) {
        unsigned long long *best = reinterpret_cast<unsigned long long *>(&acc->pad[0]);
        STATIC_CUDA(lap_launch_argmax_degree(rowinfo, n, best, st));
        unsigned long long h = 0;
        STATIC_CUDA(cudaMemcpyAsync(&h, best, sizeof(h), cudaMemcpyDeviceToHost, st));
        STATIC_CUDA(cudaStreamSynchronize(st));
        root = (int32_t)(0xFFFFFFFFu - (uint32_t)(h & 0xFFFFFFFFull));
    }
    int32_t arcs = 0;
    STATIC_CUDA(cudaMemcpyAsync(&arcs, row_ptr + n, sizeof(arcs), cudaMemcpyDeviceToHost, st));
    STATIC_CUDA(cudaStreamSynchronize(st));

    LapSampleLaunch p;
    memset(&p, 0, sizeof(p));
    p.g = LapDevGraph{rowinfo, col_idx, n, arcs};
    p.root = root;
    p.seed = seed;
    p.slots = slots;
    p.ws = state;
    p.slot_epoch = slot_epoch;
    p.rep1 = rep;
    p.cnt2 = reinterpret_cast<unsigned long long *>(cnt2);
    p.acc = acc;
    p.step_limit = (1ull << 20) + 1024ull * (uint64_t)n;
    p.num_sms = num_sms;
    // Launches of at most 2^24 samples (a launch's sample count is 32-bit);
    // each claims its ids from a counter that starts at zero.
    const uint64_t chunk = 1ull << 24;
    for (uint64_t done = 0; done < n_samples;) {
        const uint64_t c = n_samples - done < chunk ? n_samples - done : chunk;
        p.first = (uint32_t)(first_id + done);
        p.count = (uint32_t)c;
        STATIC_CUDA(cudaMemsetAsync(&acc->claim, 0, sizeof(unsigned int), st));
        STATIC_CUDA(lap_launch_sample(p, st));
        done += c;
    }
    // cnt1 = omega (first visit of every non-root node) + repeats.
    STATIC_CUDA(lap_launch_counts(n, root, n_samples, rep, reinterpret_cast<unsigned long long *>(cnt1), st));
    STATIC_CUDA(cudaMemcpyAsync(sums2, &acc->sum_y1, 2 * sizeof(uint64_t), cudaMemcpyDeviceToDevice, st));
    LapDevAcc h;
    STATIC_CUDA(cudaMemcpyAsync(&h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
    STATIC_CUDA(cudaStreamSynchronize(st));
    if (h.status & LAP_DEV_STEP_LIMIT)
        return fail_static(LAP_ERR_STEP_LIMIT, "a sample exceeded the per-sample step budget (is the graph connected?)");
    if (h.status & LAP_DEV_K_OVERFLOW)
        return fail_static(LAP_ERR_STEP_LIMIT, "a node was visited more than 2^30 times in one sample");
    if (h.status & LAP_DEV_BAD_INDEX)
        return fail_static(LAP_ERR_CUDA, "internal error: node index out of range caught in the sampler");
    g_static_error = "no error";
    return LAP_OK;
}

}  // extern "C"
