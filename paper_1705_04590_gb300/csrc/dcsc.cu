// dcsc.cu -- doubly compressed sparse column (DCSC) tiles of the adjacency
// matrix ("Graph Representation": IR row ids, JC ids of the non-empty
// columns, CP column pointers; O(nnz) storage however many tiles there are).
//
// The n vertices are cut into p blocks of B consecutive ids (p <= SM count,
// B a multiple of 32 so blocks are whole bitmap words).  Tile (i, j) holds the
// entries A(u, v) with u in block i (rows) and v in block j (columns); tiles
// are stored i-major, each as DCSC over its columns v:
//     tile_ptr[i*p + j] .. tile_ptr[i*p + j + 1]   its range of JC/CP entries
//     JC[x]        v - j*B of the x-th non-empty column, ascending
//     CP[x]..CP[x+1]   its range of IR entries
//     IR[e]        u - i*B, ascending within a column
// This is the on-chip form of the paper's 2D p_r x p_c decomposition with
// p_r = p_c = p: the search kernel (bfs_single.cu, bfs_dcsc_kernel) gives CTA
// b the rows of block b, so a top-down claim (column k of tiles (b, *)) and a
// bottom-up search (column u of tiles (*, b); the matrix is symmetric) only
// ever touch vertices that CTA owns.
//
// Build: every CSR entry (u, v) becomes the key ((i*p + j) << 2w | (v-jB) << w
// | (u-iB)) with w = bits of B; one radix sort orders the entries tile by
// tile, column by column, row by row; run boundaries of (tile, column) give
// JC/CP, a histogram of tiles gives tile_ptr.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <vector>

#include "bfs_internal.h"

namespace bfsk_dcsc {

// warp per row: keys of the row's entries at their CSR positions
__global__ void k_tile_keys(const long long* __restrict__ off, const int* __restrict__ cols, long long n,
                            long long B, int p, int w, unsigned long long* __restrict__ keys) {
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
        const long long s = off[u], e = off[u + 1];
        const long long i = u / B;
        const unsigned long long ul = (unsigned long long)(u - i * B);
        for (long long k = s + lane; k < e; k += 32) {
            const long long v = cols[k];
            const long long j = v / B;
            const unsigned long long t = (unsigned long long)(i * p + j);
            keys[k] = (t << (2 * w)) | ((unsigned long long)(v - j * B) << w) | ul;
        }
    }
}

// flag[x] = 1 where a new (tile, column) run starts; IR[x] = row within block
__global__ void k_runs(const unsigned long long* __restrict__ keys, long long nnz, int w,
                       long long* __restrict__ flag, int* __restrict__ ir) {
    const long long nth = (long long)gridDim.x * blockDim.x;
    const unsigned long long lo = (1ull << w) - 1ull;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < nnz; x += nth) {
        const unsigned long long k = keys[x];
        ir[x] = (int)(k & lo);
        flag[x] = (x == 0 || (keys[x - 1] >> w) != (k >> w)) ? 1 : 0;
    }
}

// scatter run starts: CP[pos] = x, JC[pos] = column; count runs per tile
__global__ void k_scatter_runs(const unsigned long long* __restrict__ keys, const long long* __restrict__ flag,
                               const long long* __restrict__ pos, long long nnz, int w, long long* __restrict__ cp,
                               int* __restrict__ jc, unsigned long long* __restrict__ tile_cnt) {
    const long long nth = (long long)gridDim.x * blockDim.x;
    const unsigned long long lo = (1ull << w) - 1ull;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < nnz; x += nth) {
        if (!flag[x]) continue;
        const unsigned long long k = keys[x];
        const long long y = pos[x];
        cp[y] = x;
        jc[y] = (int)((k >> w) & lo);
        atomicAdd(tile_cnt + (k >> (2 * w)), 1ull);
    }
}

__global__ void k_set_i64(long long* p, long long v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

}  // namespace bfsk_dcsc

namespace bfsrt {

using namespace bfsk_dcsc;

static int dgrid(long long items, int block, int sms) {
    long long g = (items + block - 1) / block;
    long long cap = (long long)sms * 32;
    return (int)std::max(1LL, std::min(g, cap));
}

bfs_status build_dcsc_tiles(bfs_graph* g, cudaStream_t s) {
    DcscTiles& D = g->dcsc;
    const long long n = g->n, nnz = g->nnz;
    int p = std::min<long long>((long long)g->sm_count, std::max(1LL, (n + 31) / 32));
    long long B = ((n + p - 1) / p + 31) / 32 * 32;
    p = (int)((n + B - 1) / B);
    if (B / 8 * 2 > 200 * 1024)
        return fail(BFS_ERR_UNSUPPORTED, "DCSC tiles: block of " + std::to_string(B) +
                                             " vertices does not fit two bitmaps in shared memory");
    int w = 1;
    while ((1LL << w) < B) w++;
    int tb = 1;
    while ((1LL << tb) < (long long)p * p) tb++;
    if (tb + 2 * w > 64) return fail(BFS_ERR_UNSUPPORTED, "DCSC tiles: key does not fit 64 bits");
    D.num_blocks = p;
    D.block_size = B;
    D.bits = w;
    const long long tiles = (long long)p * p;

    struct Buf {
        DeviceAlloc* m;
        cudaStream_t s;
        void* p = nullptr;
        size_t b = 0;
        Buf(DeviceAlloc* mm, cudaStream_t ss) : m(mm), s(ss) {}
        bool get(size_t bytes) { b = bytes; p = m->alloc(bytes, s); return p != nullptr; }
        ~Buf() { if (p) m->release(p, b, s); }
    };
    Buf ka(&g->mem, s), kb(&g->mem, s), flag(&g->mem, s), pos(&g->mem, s), tcnt(&g->mem, s), tmp(&g->mem, s);
    const size_t nk = (size_t)std::max(nnz, 1LL);
    if (!ka.get(8 * nk) || !kb.get(8 * nk) || !flag.get(8 * nk) || !pos.get(8 * nk) || !tcnt.get(8 * (size_t)tiles))
        return fail(BFS_ERR_OOM, "DCSC tiles: build buffers");
    D.ir = (int32_t*)g->mem.alloc(sizeof(int32_t) * (size_t)(nnz + kColPad), s);
    D.tile_ptr = (int64_t*)g->mem.alloc(sizeof(int64_t) * (size_t)(tiles + 1), s);
    if (!D.ir || !D.tile_ptr) return fail(BFS_ERR_OOM, "DCSC tiles: IR / tile pointers");
    BFS_CUDA_TRY(cudaMemsetAsync(D.ir + nnz, 0, sizeof(int32_t) * kColPad, s));
    BFS_CUDA_TRY(cudaMemsetAsync(tcnt.p, 0, 8 * (size_t)tiles, s));
    long long nzc = 0;
    if (nnz > 0) {
        k_tile_keys<<<dgrid(n * 32, 256, g->sm_count), 256, 0, s>>>((const long long*)g->offsets, g->cols, n, B, p, w,
                                                                   (unsigned long long*)ka.p);
        BFS_CUDA_TRY(cudaGetLastError());
        cub::DoubleBuffer<unsigned long long> db((unsigned long long*)ka.p, (unsigned long long*)kb.p);
        size_t tsort = 0, tscan = 0;
        BFS_CUDA_TRY(cub::DeviceRadixSort::SortKeys(nullptr, tsort, db, nnz, 0, tb + 2 * w, s));
        BFS_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, tscan, (long long*)flag.p, (long long*)pos.p, nnz, s));
        if (!tmp.get(std::max(tsort, tscan) + 256)) return fail(BFS_ERR_OOM, "DCSC tiles: sort scratch");
        BFS_CUDA_TRY(cub::DeviceRadixSort::SortKeys(tmp.p, tsort, db, nnz, 0, tb + 2 * w, s));
        const unsigned long long* sorted = db.Current();
        k_runs<<<dgrid(nnz, 256, g->sm_count), 256, 0, s>>>(sorted, nnz, w, (long long*)flag.p, D.ir);
        BFS_CUDA_TRY(cudaGetLastError());
        BFS_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp.p, tscan, (long long*)flag.p, (long long*)pos.p, nnz, s));
        long long last[2] = {0, 0};
        BFS_CUDA_TRY(cudaMemcpyAsync(&last[0], (long long*)pos.p + (nnz - 1), 8, cudaMemcpyDeviceToHost, s));
        BFS_CUDA_TRY(cudaMemcpyAsync(&last[1], (long long*)flag.p + (nnz - 1), 8, cudaMemcpyDeviceToHost, s));
        BFS_CUDA_TRY(cudaStreamSynchronize(s));
        nzc = last[0] + last[1];
        D.jc = (int32_t*)g->mem.alloc(sizeof(int32_t) * (size_t)std::max(nzc, 1LL), s);
        D.cp = (int64_t*)g->mem.alloc(sizeof(int64_t) * (size_t)(nzc + 1), s);
        if (!D.jc || !D.cp) return fail(BFS_ERR_OOM, "DCSC tiles: JC / CP");
        k_scatter_runs<<<dgrid(nnz, 256, g->sm_count), 256, 0, s>>>(sorted, (const long long*)flag.p,
                                                                   (const long long*)pos.p, nnz, w, (long long*)D.cp,
                                                                   D.jc, (unsigned long long*)tcnt.p);
        BFS_CUDA_TRY(cudaGetLastError());
        k_set_i64<<<1, 32, 0, s>>>((long long*)D.cp + nzc, nnz);
        BFS_CUDA_TRY(cudaGetLastError());
    } else {
        D.jc = (int32_t*)g->mem.alloc(sizeof(int32_t), s);
        D.cp = (int64_t*)g->mem.alloc(sizeof(int64_t), s);
        if (!D.jc || !D.cp) return fail(BFS_ERR_OOM, "DCSC tiles: JC / CP");
        BFS_CUDA_TRY(cudaMemsetAsync(D.cp, 0, sizeof(int64_t), s));
    }
    // tile pointers: exclusive scan of runs per tile (p^2 entries; host side)
    std::vector<unsigned long long> cnt((size_t)tiles);
    BFS_CUDA_TRY(cudaMemcpyAsync(cnt.data(), tcnt.p, 8 * (size_t)tiles, cudaMemcpyDeviceToHost, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<int64_t> tp((size_t)tiles + 1, 0);
    for (long long t = 0; t < tiles; t++) tp[(size_t)t + 1] = tp[(size_t)t] + (int64_t)cnt[(size_t)t];
    if (tp[(size_t)tiles] != nzc) return fail(BFS_ERR_CUDA, "DCSC tiles: run count mismatch (internal)");
    BFS_CUDA_TRY(cudaMemcpyAsync(D.tile_ptr, tp.data(), 8 * (size_t)(tiles + 1), cudaMemcpyHostToDevice, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    D.nzc = nzc;
    D.bytes = sizeof(int32_t) * (size_t)(nnz + kColPad) + sizeof(int64_t) * (size_t)(tiles + 1) +
              sizeof(int32_t) * (size_t)std::max(nzc, 1LL) + sizeof(int64_t) * (size_t)(nzc + 1);
    D.built = true;
    return BFS_OK;
}

void release_dcsc_tiles(bfs_graph* g) {
    DcscTiles& D = g->dcsc;
    if (!D.built) return;
    g->mem.release(D.ir, sizeof(int32_t) * (size_t)(g->nnz + kColPad), nullptr);
    g->mem.release(D.tile_ptr, sizeof(int64_t) * (size_t)((long long)D.num_blocks * D.num_blocks + 1), nullptr);
    g->mem.release(D.jc, sizeof(int32_t) * (size_t)std::max(D.nzc, 1LL), nullptr);
    g->mem.release(D.cp, sizeof(int64_t) * (size_t)(D.nzc + 1), nullptr);
    D = DcscTiles();
}

}  // namespace bfsrt
