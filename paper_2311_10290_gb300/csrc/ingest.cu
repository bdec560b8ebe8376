// Graph ingest on the GPU (hot-path row a1; cold, once per graph):
// CSR validation against the graph model of Section 2 (undirected, simple),
// per-node row records, the landmark choice of Section 6 (highest degree,
// smallest id on ties) and a breadth-first search from the landmark that
// checks connectivity (Section 2 assumes G connected; Wilson's algorithm does
// not terminate otherwise) and records hop distances.
#include "lap_internal.h"

namespace {

constexpr int kBlock = 256;

int grid_for(int64_t work, int block)
{
    int64_t g = (work + block - 1) / block;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

__device__ __forceinline__ bool row_contains(const int32_t *col, int32_t a, int32_t b, int32_t x)
{
    // Rows are checked to be strictly ascending, so binary search applies.
    while (a < b) {
        int32_t mid = a + ((b - a) >> 1);
        int32_t y = col[mid];
        if (y == x) return true;
        if (y < x) a = mid + 1; else b = mid;
    }
    return false;
}

__global__ void validate_kernel(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                int32_t n, int64_t arcs, unsigned int *status)
{
    unsigned int bad = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = row_ptr[u], b = row_ptr[u + 1];
        if (a < 0 || b < a || (int64_t)b > arcs) { bad |= LAP_DEV_BAD_CSR; continue; }
        for (int32_t e = a; e < b; ++e) {
            int32_t w = col[e];
            if (w < 0 || w >= n) { bad |= LAP_DEV_BAD_CSR; continue; }
            if (w == (int32_t)u) bad |= LAP_DEV_SELF_LOOP;
            if (e > a && col[e - 1] >= w) bad |= LAP_DEV_BAD_CSR;
        }
    }
    if (bad) atomicOr(status, bad);
}

// Symmetry needs sorted rows, so it runs after validate_kernel succeeded.
__global__ void symmetry_kernel(const int32_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                int32_t n, unsigned int *status)
{
    unsigned int bad = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = row_ptr[u], b = row_ptr[u + 1];
        for (int32_t e = a; e < b; ++e) {
            int32_t w = col[e];
            if (!row_contains(col, row_ptr[w], row_ptr[w + 1], (int32_t)u)) { bad |= LAP_DEV_NOT_SYMMETRIC; break; }
        }
    }
    if (bad) atomicOr(status, bad);
}

__global__ void rowinfo_kernel(const int32_t *__restrict__ row_ptr, int32_t n, int2 *__restrict__ rowinfo)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = row_ptr[u];
        rowinfo[u] = make_int2(a, row_ptr[u + 1] - a);
    }
}

// Packs (degree, ~id) so that the maximum is the highest degree with the
// smallest id among ties.
__global__ void argmax_degree_kernel(const int2 *__restrict__ rowinfo, int32_t n, unsigned long long *best)
{
    unsigned long long m = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long key = ((unsigned long long)(uint32_t)rowinfo[u].y << 32) | (0xFFFFFFFFu - (uint32_t)u);
        m = key > m ? key : m;
    }
    for (int off = 16; off > 0; off >>= 1) {
        unsigned long long o = __shfl_down_sync(0xFFFFFFFFu, m, off);
        m = o > m ? o : m;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(best, m);
}

__global__ void bfs_init_kernel(int32_t *hops, int32_t n, int32_t root)
{
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        hops[u] = (u == root) ? 0 : -1;
}

__global__ void bfs_level_kernel(const int2 *__restrict__ rowinfo, const int32_t *__restrict__ col,
                                 int32_t *hops, int32_t n, int32_t level, unsigned int *found)
{
    unsigned int got = 0;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        if (hops[u] != level) continue;
        int2 r = rowinfo[u];
        for (int32_t e = 0; e < r.y; ++e) {
            int32_t w = col[r.x + e];
            if (atomicCAS(&hops[w], -1, level + 1) == -1) ++got;
        }
    }
    if (got) atomicAdd(found, got);
}

}  // namespace

cudaError_t lap_launch_validate(const int32_t *row_ptr, const int32_t *col, int32_t n, int64_t arcs,
                                unsigned int *status, cudaStream_t st)
{
    validate_kernel<<<grid_for(n, kBlock), kBlock, 0, st>>>(row_ptr, col, n, arcs, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    unsigned int h = 0;
    if ((e = cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
    if (h & LAP_DEV_BAD_CSR) return cudaSuccess;     // symmetry search needs a well-formed CSR
    symmetry_kernel<<<grid_for(n, kBlock), kBlock, 0, st>>>(row_ptr, col, n, status);
    return cudaGetLastError();
}

cudaError_t lap_launch_rowinfo(const int32_t *row_ptr, int32_t n, int2 *rowinfo, cudaStream_t st)
{
    rowinfo_kernel<<<grid_for(n, kBlock), kBlock, 0, st>>>(row_ptr, n, rowinfo);
    return cudaGetLastError();
}

cudaError_t lap_launch_argmax_degree(const int2 *rowinfo, int32_t n, unsigned long long *best, cudaStream_t st)
{
    argmax_degree_kernel<<<grid_for(n, kBlock), kBlock, 0, st>>>(rowinfo, n, best);
    return cudaGetLastError();
}

cudaError_t lap_launch_bfs_init(int32_t *hops, int32_t n, int32_t root, cudaStream_t st)
{
    bfs_init_kernel<<<grid_for(n, kBlock), kBlock, 0, st>>>(hops, n, root);
    return cudaGetLastError();
}

cudaError_t lap_launch_bfs_level(const int2 *rowinfo, const int32_t *col, int32_t *hops, int32_t n,
                                 int32_t level, unsigned int *found, cudaStream_t st)
{
    bfs_level_kernel<<<grid_for(n, kBlock), kBlock, 0, st>>>(rowinfo, col, hops, n, level, found);
    return cudaGetLastError();
}
