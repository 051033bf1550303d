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
//
// Beside the rows sit their heads: per vertex its degree and the first seven
// ids of its reordered row, one aligned 32-byte record (one DRAM sector).  A
// bottom-up sweep reads them in vertex order (one coalesced stream, no offsets
// lookup in front of a scattered row read) and goes to the full row only for
// the few searchers whose first seven neighbours are all outside the frontier.
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

// heads[2u] = {deg(u), r0, r1, r2}, heads[2u + 1] = {r3, r4, r5, r6}: the first
// seven ids of u's reordered row, 0 past its end; first[u] = r0 | (deg(u) >= 2)
// << 31 (the plane a bottom-up sweep streams: its first probe, and whether the
// row goes on); one thread per vertex, first[] zero-padded to n + 32
__global__ void k_hub_heads(const long long* __restrict__ off, const int32_t* __restrict__ cols_hf, long long n,
                            int4* __restrict__ heads, int32_t* __restrict__ first) {
    const long long nth = (long long)gridDim.x * blockDim.x;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n + 32; u += nth) {
        if (u >= n) {
            first[u] = 0;
            continue;
        }
        const long long s = off[u], dg = off[u + 1] - s;
        int r[7];
#pragma unroll
        for (int t = 0; t < 7; t++) r[t] = t < dg ? cols_hf[s + t] : 0;
        heads[2 * u] = make_int4((int)dg, r[0], r[1], r[2]);
        heads[2 * u + 1] = make_int4(r[3], r[4], r[5], r[6]);
        first[u] = (int32_t)((unsigned)r[0] | (dg >= 2 ? 0x80000000u : 0u));
    }
}

}  // namespace bfsk_hub

namespace bfsrt {

using namespace bfsk_hub;

static bfs_status build_bu_heads(bfs_graph* g, cudaStream_t s) {
    const long long n = g->n;
    const size_t bytes = sizeof(int32_t) * 8 * (size_t)n;
    const size_t fbytes = sizeof(int32_t) * (size_t)(n + 32);
    g->bu_heads = (int32_t*)g->mem.alloc(bytes, s);
    g->bu_first = (int32_t*)g->mem.alloc(fbytes, s);
    if (!g->bu_heads || !g->bu_first) {
        if (g->bu_heads) g->mem.release(g->bu_heads, bytes, s);
        if (g->bu_first) g->mem.release(g->bu_first, fbytes, s);
        g->bu_heads = nullptr;
        g->bu_first = nullptr;
        return fail(BFS_ERR_OOM, "hub-first rows: row heads");
    }
    const int blocks = std::max(1, std::min<int>(g->sm_count * 8, (int)((n + 32 + 255) / 256)));
    k_hub_heads<<<blocks, 256, 0, s>>>((const long long*)g->offsets, g->cols_hf, n,
                                       reinterpret_cast<int4*>(g->bu_heads), g->bu_first);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        g->mem.release(g->bu_heads, bytes, s);
        g->mem.release(g->bu_first, fbytes, s);
        g->bu_heads = nullptr;
        g->bu_first = nullptr;
        return cuda_fail(e, "hub-first rows: row heads");
    }
    g->graph_bytes += bytes + fbytes;
    return BFS_OK;
}

bfs_status build_hub_first_rows(bfs_graph* g, cudaStream_t s) {
    if (g->cols_hf) return BFS_OK;
    const long long n = g->n, nnz = g->nnz;
    g->cols_hf = (int32_t*)g->mem.alloc(sizeof(int32_t) * (size_t)(nnz + kColPad), s);
    if (!g->cols_hf) return fail(BFS_ERR_OOM, "hub-first rows: column copy");
    BFS_CUDA_TRY(cudaMemsetAsync(g->cols_hf + nnz, 0, sizeof(int32_t) * kColPad, s));
    if (nnz == 0) {
        g->graph_bytes += sizeof(int32_t) * (size_t)(nnz + kColPad);
        return build_bu_heads(g, s);
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
    return build_bu_heads(g, s);
}

}  // namespace bfsrt
