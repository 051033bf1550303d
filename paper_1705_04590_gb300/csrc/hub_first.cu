// hub_first.cu -- second copy of the column ids with every row ordered by
// neighbour degree, highest first (ties by id, ascending); graph build, off
// the timed path.
//
// Algorithm 2 scans a vertex's neighbours in stored order and stops at the
// first one in the frontier; the paper stores rows sorted by id.  Any order
// finds a valid parent at the same level; putting high-degree neighbours
// first makes the first probe hit far more often on R-MAT graphs, whose
// frontiers near the dense levels are made of high-degree vertices.  The top-
// down direction keeps the id-sorted rows.
//
// Built with one stable radix sort of (row, ~degree(neighbour)) keys carrying
// the neighbour ids: within a row, equal degrees keep the id order of the
// input rows.
#include <cub/device/device_radix_sort.cuh>

#include "bfs_internal.h"

namespace bfsk_hub {

// keys[k] = row(k) << 32 | (2^32 - 1 - deg(cols[k])), one warp per row
__global__ void k_hub_keys(const long long* __restrict__ off, const int32_t* __restrict__ cols, long long n,
                           unsigned long long* __restrict__ keys) {
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
        const long long s = off[u], e = off[u + 1];
        for (long long k = s + lane; k < e; k += 32) {
            const int v = cols[k];
            const long long dv = off[v + 1] - off[v];
            const unsigned inv = 0xFFFFFFFFu - (unsigned)(dv > 0xFFFFFFFFLL ? 0xFFFFFFFFLL : dv);
            keys[k] = ((unsigned long long)u << 32) | inv;
        }
    }
}

}  // namespace bfsk_hub

namespace bfsrt {

using namespace bfsk_hub;

bfs_status build_hub_first_rows(bfs_graph* g, cudaStream_t s) {
    if (g->cols_hf) return BFS_OK;
    const long long n = g->n, nnz = g->nnz;
    g->cols_hf = (int32_t*)g->mem.alloc(sizeof(int32_t) * (size_t)(nnz + kColPad), s);
    if (!g->cols_hf) return fail(BFS_ERR_OOM, "hub-first rows: column copy");
    BFS_CUDA_TRY(cudaMemsetAsync(g->cols_hf + nnz, 0, sizeof(int32_t) * kColPad, s));
    if (nnz == 0) {
        g->graph_bytes += sizeof(int32_t) * (size_t)(nnz + kColPad);
        return BFS_OK;
    }
    int end_bit = 32;
    while ((1LL << (end_bit - 32)) < n) end_bit++;
    unsigned long long* k0 = (unsigned long long*)g->mem.alloc(sizeof(unsigned long long) * (size_t)nnz, s);
    unsigned long long* k1 = (unsigned long long*)g->mem.alloc(sizeof(unsigned long long) * (size_t)nnz, s);
    int32_t* v1 = (int32_t*)g->mem.alloc(sizeof(int32_t) * (size_t)nnz, s);
    auto release = [&]() {
        if (k0) g->mem.release(k0, sizeof(unsigned long long) * (size_t)nnz, s);
        if (k1) g->mem.release(k1, sizeof(unsigned long long) * (size_t)nnz, s);
        if (v1) g->mem.release(v1, sizeof(int32_t) * (size_t)nnz, s);
    };
    if (!k0 || !k1 || !v1) {
        release();
        g->mem.release(g->cols_hf, sizeof(int32_t) * (size_t)(nnz + kColPad), s);
        g->cols_hf = nullptr;
        return fail(BFS_ERR_OOM, "hub-first rows: sort buffers");
    }
    const int blocks = std::max(1, std::min<int>(g->sm_count * 16, (int)((n + 7) / 8)));
    k_hub_keys<<<blocks, 256, 0, s>>>((const long long*)g->offsets, g->cols, n, k0);
    cudaError_t e = cudaGetLastError();
    // values start as the id-sorted column copy; the sort is stable
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->cols_hf, g->cols, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToDevice, s);
    cub::DoubleBuffer<unsigned long long> kb(k0, k1);
    cub::DoubleBuffer<int32_t> vb(g->cols_hf, v1);
    size_t tb = 0;
    if (e == cudaSuccess) e = cub::DeviceRadixSort::SortPairs(nullptr, tb, kb, vb, (int64_t)nnz, 0, end_bit, s);
    void* tmp = nullptr;
    if (e == cudaSuccess) {
        tmp = g->mem.alloc(tb + 16, s);
        if (!tmp) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess) e = cub::DeviceRadixSort::SortPairs(tmp, tb, kb, vb, (int64_t)nnz, 0, end_bit, s);
    if (e == cudaSuccess && vb.Current() != g->cols_hf)
        e = cudaMemcpyAsync(g->cols_hf, vb.Current(), sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (tmp) g->mem.release(tmp, tb + 16, s);
    release();
    if (e != cudaSuccess) {
        g->mem.release(g->cols_hf, sizeof(int32_t) * (size_t)(nnz + kColPad), s);
        g->cols_hf = nullptr;
        return cuda_fail(e, "hub-first rows: sort");
    }
    g->graph_bytes += sizeof(int32_t) * (size_t)(nnz + kColPad);
    return BFS_OK;
}

}  // namespace bfsrt
