// graph_build.cu -- device-side graph construction (off the timed path).
//
// "Graph Representation": adjacencies of each vertex sorted and stored
// contiguously, every undirected edge stored in both rows, an n+1 row
// pointer array (64-bit here; column ids 32-bit).  "Data Sets": duplicate
// edges pruned.  Self-loops are dropped as well.
//
// Edge list -> CSR: each edge {u, v}, u != v, becomes the 64-bit keys
// (u << 32 | v) and (v << 32 | u); the keys are radix-sorted (CUB) and
// de-duplicated; the low halves are the column ids and a degree count plus
// an exclusive scan gives the row offsets.  A directed graph ("Data Sets":
// the method applies to directed graphs) keeps only (u << 32 | v) for the
// out-edge CSR and builds its transpose the same way from (v << 32 | u): the
// in-edge rows the bottom-up step scans.  Also built here: the bitmap of
// vertices that never search (no edge into them, or ids past n in the last
// word).
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cub/device/device_select.cuh>

#include "bfs_internal.h"

namespace bfsk_build {

__global__ void k_check_and_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, long long m,
                                 long long n, int symmetric, unsigned long long* __restrict__ keys,
                                 unsigned long long* __restrict__ count, int* __restrict__ bad) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long nth = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + threadIdx.x - lane; base < m; base += nth) {
        const long long i = base + lane;
        bool keep = false;
        unsigned long long k0 = 0, k1 = 0;
        if (i < m) {
            const int u = src[i], v = dst[i];
            if (u < 0 || v < 0 || (long long)u >= n || (long long)v >= n) {
                atomicExch(bad, 1);
            } else if (u != v) {
                keep = true;
                k0 = ((unsigned long long)(unsigned)u << 32) | (unsigned)v;
                k1 = ((unsigned long long)(unsigned)v << 32) | (unsigned)u;
            }
        }
        const unsigned km = __ballot_sync(full, keep);
        if (km) {
            const int leader = __ffs(km) - 1;
            unsigned long long b = 0;
            const unsigned long long per = symmetric ? 2ull : 1ull;
            if (lane == leader) b = atomicAdd(count, per * __popc(km));
            b = __shfl_sync(full, b, leader);
            if (keep) {
                unsigned lt;
                asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
                const unsigned long long pos = b + per * __popc(km & lt);
                keys[pos] = k0;
                if (symmetric) keys[pos + 1] = k1;
            }
        }
    }
}

__global__ void k_split_keys(const unsigned long long* __restrict__ keys, long long nnz, int32_t* __restrict__ cols,
                             unsigned long long* __restrict__ deg) {
    const long long nth = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += nth) {
        const unsigned long long k = keys[i];
        cols[i] = (int32_t)(k & 0xffffffffull);
        atomicAdd(deg + (k >> 32), 1ull);
    }
}

__global__ void k_fill_i32(int32_t* p, long long cnt, int32_t v) {
    const long long nth = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += nth) p[i] = v;
}

__global__ void k_isolated(const long long* __restrict__ off, long long n, long long W, uint32_t* __restrict__ iso) {
    const long long nth = (long long)gridDim.x * blockDim.x;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < W; w += nth) {
        uint32_t x = 0;
        for (int b = 0; b < 32; b++) {
            const long long v = w * 32 + b;
            if (v >= n || off[v + 1] == off[v]) x |= 1u << b;
        }
        iso[w] = x;
    }
}

// 64-bit endpoints narrowed to int32; *bad = 1 when one lies outside [0, n)
__global__ void k_narrow_edges(const int64_t* __restrict__ s64, const int64_t* __restrict__ d64, long long m,
                               long long n, int32_t* __restrict__ s32, int32_t* __restrict__ d32, int* bad) {
    const long long nth = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += nth) {
        const int64_t a = s64[i], b = d64[i];
        if (a < 0 || a >= n || b < 0 || b >= n) {
            *bad = 1;
            s32[i] = 0;
            d32[i] = 0;
        } else {
            s32[i] = (int32_t)a;
            d32[i] = (int32_t)b;
        }
    }
}

// number of vertices with degree > 0 (clear bits of the isolated bitmap)
__global__ void k_count_active(const uint32_t* __restrict__ iso, long long W, unsigned long long* cnt) {
    const long long nth = (long long)gridDim.x * blockDim.x;
    unsigned long long c = 0;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < W; w += nth) c += __popc(~iso[w]);
    if (c) atomicAdd(cnt, c);
}

// deg8[v] = min(deg(v), 255): the degree as bottom-up and top-down steps need it
// (a coalesced byte stream instead of two int64 offsets per vertex); and the
// largest degree into *dmax
__global__ void k_deg8(const long long* __restrict__ off, long long n, uint8_t* __restrict__ deg8,
                       unsigned long long* dmax) {
    const long long nth = (long long)gridDim.x * blockDim.x;
    unsigned long long mx = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n + 32; v += nth) {
        const long long dg = v < n ? off[v + 1] - off[v] : 0;
        deg8[v] = (uint8_t)(dg < 255 ? dg : 255);
        mx = dg > (long long)mx ? (unsigned long long)dg : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = t > mx ? t : mx;
    }
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(dmax, mx);
}

// CSR validation: warp per row.  bad codes: 1 offsets, 2 id range, 3 order/duplicate, 4 self-loop, 5 asymmetric
__global__ void k_check_csr(const long long* __restrict__ off, const int32_t* __restrict__ cols, long long n,
                            long long nnz, int check_sym, int* __restrict__ bad) {
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long r = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5); r < n; r += nw) {
        const long long s = off[r], e = off[r + 1];
        if (s > e || s < 0 || e > nnz) {
            if (lane == 0) atomicMax(bad, 1);
            continue;
        }
        for (long long k = s + lane; k < e; k += 32) {
            const int c = cols[k];
            if (c < 0 || (long long)c >= n) { atomicMax(bad, 2); continue; }
            if (c == (int)r) atomicMax(bad, 4);
            if (k + 1 < e && !(c < cols[k + 1])) atomicMax(bad, 3);
            if (check_sym) {
                long long lo = off[c], hi = off[c + 1];
                if (lo < 0 || hi > nnz || lo > hi) { atomicMax(bad, 1); continue; }
                while (lo < hi) {
                    const long long mid = lo + (hi - lo) / 2;
                    if (cols[mid] < (int)r) lo = mid + 1; else hi = mid;
                }
                if (lo >= off[c + 1] || cols[lo] != (int)r) atomicMax(bad, 5);
            }
        }
    }
}

}  // namespace bfsk_build

namespace bfsrt {

using namespace bfsk_build;

static int grid_for(long long items, int block, int sms) {
    long long g = (items + block - 1) / block;
    long long cap = (long long)sms * 32;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// RAII scratch through the graph's allocator
struct Scratch {
    DeviceAlloc* mem;
    cudaStream_t s;
    void* p = nullptr;
    size_t bytes = 0;
    Scratch(DeviceAlloc* m, cudaStream_t st) : mem(m), s(st) {}
    bool get(size_t b) {
        p = mem->alloc(b, s);
        bytes = b;
        return p != nullptr;
    }
    ~Scratch() {
        if (p) mem->release(p, bytes, s);
    }
};

static bfs_status finish_offsets(bfs_graph* g, int64_t* offsets, unsigned long long* deg, cudaStream_t s) {
    // offsets[0] = 0, offsets[1..n] = inclusive scan of degrees
    const long long n = g->n;
    size_t tb = 0;
    BFS_CUDA_TRY(cub::DeviceScan::InclusiveSum(nullptr, tb, deg, (unsigned long long*)offsets + 1, n, s));
    Scratch tmp(&g->mem, s);
    if (!tmp.get(tb + 16)) return fail(BFS_ERR_OOM, "graph build: scan scratch");
    BFS_CUDA_TRY(cudaMemsetAsync(offsets, 0, sizeof(int64_t), s));
    BFS_CUDA_TRY(cub::DeviceScan::InclusiveSum(tmp.p, tb, deg, (unsigned long long*)offsets + 1, n, s));
    return BFS_OK;
}

bfs_status build_isolated_bitmap(bfs_graph* g, cudaStream_t s) {
    g->W = (g->n + 31) / 32;
    g->isolated = (uint32_t*)g->mem.alloc(sizeof(uint32_t) * (size_t)g->W, s);
    if (!g->isolated) return fail(BFS_ERR_OOM, "graph build: isolated bitmap");
    g->graph_bytes += sizeof(uint32_t) * (size_t)g->W;
    // vertices no edge leads into never search bottom-up and are never reached (but a root)
    const int64_t* rows_in = g->directed ? g->offsets_in : g->offsets;
    k_isolated<<<grid_for(g->W, 256, g->sm_count), 256, 0, s>>>((const long long*)rows_in, g->n, g->W,
                                                                g->isolated);
    BFS_CUDA_TRY(cudaGetLastError());
    {
        Scratch cnt(&g->mem, s);
        if (!cnt.get(16)) return fail(BFS_ERR_OOM, "graph build: counter");
        BFS_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, 16, s));
        k_count_active<<<grid_for(g->W, 256, g->sm_count), 256, 0, s>>>(g->isolated, g->W,
                                                                        (unsigned long long*)cnt.p);
        BFS_CUDA_TRY(cudaGetLastError());
        unsigned long long h = 0;
        BFS_CUDA_TRY(cudaMemcpyAsync(&h, cnt.p, sizeof h, cudaMemcpyDeviceToHost, s));
        BFS_CUDA_TRY(cudaStreamSynchronize(s));
        g->n_active = (int64_t)h;
    }
    g->deg8 = (uint8_t*)g->mem.alloc((size_t)g->n + 32, s);
    if (!g->deg8) return fail(BFS_ERR_OOM, "graph build: degree bytes");
    g->graph_bytes += (size_t)g->n + 32;
    Scratch dm(&g->mem, s);
    if (!dm.get(16)) return fail(BFS_ERR_OOM, "graph build: counter");
    BFS_CUDA_TRY(cudaMemsetAsync(dm.p, 0, 16, s));
    unsigned long long* dmax = (unsigned long long*)dm.p;
    k_deg8<<<grid_for(g->n + 32, 256, g->sm_count), 256, 0, s>>>((const long long*)g->offsets, g->n, g->deg8,
                                                                 dmax);
    BFS_CUDA_TRY(cudaGetLastError());
    if (g->directed) {
        g->deg8_in = (uint8_t*)g->mem.alloc((size_t)g->n + 32, s);
        if (!g->deg8_in) return fail(BFS_ERR_OOM, "graph build: in-degree bytes");
        g->graph_bytes += (size_t)g->n + 32;
        k_deg8<<<grid_for(g->n + 32, 256, g->sm_count), 256, 0, s>>>((const long long*)g->offsets_in, g->n,
                                                                     g->deg8_in, dmax + 1);
        BFS_CUDA_TRY(cudaGetLastError());
    }
    unsigned long long h[2] = {0, 0};
    BFS_CUDA_TRY(cudaMemcpyAsync(h, dmax, sizeof h, cudaMemcpyDeviceToHost, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    g->max_degree = (int64_t)(h[0] > h[1] ? h[0] : h[1]);
    return BFS_OK;
}

// One CSR from device edge arrays: rows of (es[i] -> ed[i]), and of (ed[i] -> es[i])
// too when symmetric; self-loops dropped, duplicates removed, rows sorted.
static bfs_status build_rows(bfs_graph* g, const int32_t* es, const int32_t* ed, int64_t m, bool symmetric,
                             int64_t** off_out, int32_t** cols_out, long long* nnz_out, cudaStream_t s) {
    const long long n = g->n;
    const long long cap = (symmetric ? 2 : 1) * (long long)m;
    Scratch keys_a(&g->mem, s), keys_b(&g->mem, s), small(&g->mem, s);
    if (!small.get(64)) return fail(BFS_ERR_OOM, "graph build: counters");
    unsigned long long* d_count = (unsigned long long*)small.p;
    int* d_bad = (int*)((char*)small.p + 16);
    unsigned long long* d_sel = (unsigned long long*)((char*)small.p + 32);
    BFS_CUDA_TRY(cudaMemsetAsync(small.p, 0, 64, s));
    if (cap > 0) {
        if (!keys_a.get(sizeof(unsigned long long) * (size_t)cap) || !keys_b.get(sizeof(unsigned long long) * (size_t)cap))
            return fail(BFS_ERR_OOM, "graph build: key buffers");
        k_check_and_keys<<<grid_for(m, 256, g->sm_count), 256, 0, s>>>(es, ed, m, n, symmetric ? 1 : 0,
                                                                      (unsigned long long*)keys_a.p, d_count, d_bad);
        BFS_CUDA_TRY(cudaGetLastError());
    }
    unsigned long long h[2] = {0, 0};
    int hbad = 0;
    BFS_CUDA_TRY(cudaMemcpyAsync(&h[0], d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    BFS_CUDA_TRY(cudaMemcpyAsync(&hbad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad) return fail(BFS_ERR_INVALID, "edge list holds a vertex id outside [0, n_vertices)");
    const long long nk = (long long)h[0];
    int end_bit = 32;
    while (end_bit < 64 && (1ll << (end_bit - 32)) < n) end_bit++;
    long long nnz = 0;
    unsigned long long* uniq = nullptr;
    if (nk > 0) {
        size_t tb = 0;
        cub::DoubleBuffer<unsigned long long> db((unsigned long long*)keys_a.p, (unsigned long long*)keys_b.p);
        BFS_CUDA_TRY(cub::DeviceRadixSort::SortKeys(nullptr, tb, db, nk, 0, end_bit, s));
        size_t tu = 0;
        BFS_CUDA_TRY(cub::DeviceSelect::Unique(nullptr, tu, (unsigned long long*)keys_a.p,
                                               (unsigned long long*)keys_b.p, d_sel, nk, s));
        Scratch tmp(&g->mem, s);
        if (!tmp.get((tb > tu ? tb : tu) + 256)) return fail(BFS_ERR_OOM, "graph build: sort scratch");
        BFS_CUDA_TRY(cub::DeviceRadixSort::SortKeys(tmp.p, tb, db, nk, 0, end_bit, s));
        unsigned long long* sorted = db.Current();
        uniq = db.Alternate();
        BFS_CUDA_TRY(cub::DeviceSelect::Unique(tmp.p, tu, sorted, uniq, d_sel, nk, s));
        BFS_CUDA_TRY(cudaMemcpyAsync(&h[1], d_sel, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        BFS_CUDA_TRY(cudaStreamSynchronize(s));
        nnz = (long long)h[1];
    }
    *nnz_out = nnz;
    *off_out = (int64_t*)g->mem.alloc(sizeof(int64_t) * (size_t)(n + 1), s);
    *cols_out = (int32_t*)g->mem.alloc(sizeof(int32_t) * (size_t)(nnz + kColPad), s);
    if (!*off_out || !*cols_out) return fail(BFS_ERR_OOM, "graph build: CSR arrays");
    g->graph_bytes += sizeof(int64_t) * (size_t)(n + 1) + sizeof(int32_t) * (size_t)(nnz + kColPad);
    Scratch deg(&g->mem, s);
    if (!deg.get(sizeof(unsigned long long) * (size_t)n)) return fail(BFS_ERR_OOM, "graph build: degrees");
    BFS_CUDA_TRY(cudaMemsetAsync(deg.p, 0, sizeof(unsigned long long) * (size_t)n, s));
    k_fill_i32<<<1, 32, 0, s>>>(*cols_out + nnz, kColPad, 0);
    BFS_CUDA_TRY(cudaGetLastError());
    if (nnz > 0) {
        k_split_keys<<<grid_for(nnz, 256, g->sm_count), 256, 0, s>>>(uniq, nnz, *cols_out, (unsigned long long*)deg.p);
        BFS_CUDA_TRY(cudaGetLastError());
    }
    return finish_offsets(g, *off_out, (unsigned long long*)deg.p, s);
}

bfs_status build_csr_from_edges(bfs_graph* g, const int32_t* src, const int32_t* dst, int64_t m, bool device_ptrs,
                                cudaStream_t s) {
    Scratch dsrc(&g->mem, s), ddst(&g->mem, s);
    const int32_t* es = src;
    const int32_t* ed = dst;
    if (!device_ptrs && m > 0) {
        if (!dsrc.get(sizeof(int32_t) * (size_t)m) || !ddst.get(sizeof(int32_t) * (size_t)m))
            return fail(BFS_ERR_OOM, "graph build: edge staging");
        BFS_CUDA_TRY(cudaMemcpyAsync(dsrc.p, src, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
        BFS_CUDA_TRY(cudaMemcpyAsync(ddst.p, dst, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
        es = (const int32_t*)dsrc.p;
        ed = (const int32_t*)ddst.p;
    }
    g->graph_bytes = 0;
    long long nnz = 0;
    bfs_status st = build_rows(g, es, ed, m, !g->directed, &g->offsets, &g->cols, &nnz, s);
    if (st != BFS_OK) return st;
    g->nnz = nnz;
    if (g->directed) {
        long long nnz_in = 0;
        st = build_rows(g, ed, es, m, false, &g->offsets_in, &g->cols_in, &nnz_in, s);
        if (st != BFS_OK) return st;
        if (nnz_in != nnz) return fail(BFS_ERR_CUDA, "graph build: transpose holds a different edge count");
    }
    st = build_isolated_bitmap(g, s);
    if (st != BFS_OK) return st;
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    return BFS_OK;
}

bfs_status build_csr_from_edges64(bfs_graph* g, const int64_t* src, const int64_t* dst, int64_t m, bool device_ptrs,
                                  cudaStream_t s) {
    Scratch s32(&g->mem, s), d32(&g->mem, s), flag(&g->mem, s), stage(&g->mem, s);
    if (m > 0 && (!s32.get(sizeof(int32_t) * (size_t)m) || !d32.get(sizeof(int32_t) * (size_t)m)))
        return fail(BFS_ERR_OOM, "graph build: int32 edge arrays");
    if (!flag.get(16)) return fail(BFS_ERR_OOM, "graph build: counter");
    BFS_CUDA_TRY(cudaMemsetAsync(flag.p, 0, 16, s));
    int* d_bad = (int*)flag.p;
    if (device_ptrs) {
        if (m > 0) {
            k_narrow_edges<<<grid_for(m, 256, g->sm_count), 256, 0, s>>>(src, dst, m, g->n, (int32_t*)s32.p,
                                                                       (int32_t*)d32.p, d_bad);
            BFS_CUDA_TRY(cudaGetLastError());
        }
    } else if (m > 0) {
        // host arrays: copied in chunks through a device staging buffer, narrowed there
        const long long chunk = std::min<long long>(m, 1LL << 24);
        if (!stage.get(2 * sizeof(int64_t) * (size_t)chunk)) return fail(BFS_ERR_OOM, "graph build: edge staging");
        int64_t* st_s = (int64_t*)stage.p;
        int64_t* st_d = st_s + chunk;
        for (long long a = 0; a < m; a += chunk) {
            const long long c = std::min(chunk, m - a);
            BFS_CUDA_TRY(cudaMemcpyAsync(st_s, src + a, sizeof(int64_t) * (size_t)c, cudaMemcpyHostToDevice, s));
            BFS_CUDA_TRY(cudaMemcpyAsync(st_d, dst + a, sizeof(int64_t) * (size_t)c, cudaMemcpyHostToDevice, s));
            k_narrow_edges<<<grid_for(c, 256, g->sm_count), 256, 0, s>>>(st_s, st_d, c, g->n, (int32_t*)s32.p + a,
                                                                       (int32_t*)d32.p + a, d_bad);
            BFS_CUDA_TRY(cudaGetLastError());
        }
    }
    int hbad = 0;
    BFS_CUDA_TRY(cudaMemcpyAsync(&hbad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad) return fail(BFS_ERR_INVALID, "an edge endpoint lies outside [0, n_vertices)");
    return build_csr_from_edges(g, (const int32_t*)s32.p, (const int32_t*)d32.p, m, true, s);
}

bfs_status build_csr_from_csr(bfs_graph* g, const int64_t* off, const int32_t* cols, bool device_ptrs,
                              bool check_symmetry, cudaStream_t s) {
    const long long n = g->n, nnz = g->nnz;
    g->offsets = (int64_t*)g->mem.alloc(sizeof(int64_t) * (size_t)(n + 1), s);
    g->cols = (int32_t*)g->mem.alloc(sizeof(int32_t) * (size_t)(nnz + kColPad), s);
    if (!g->offsets || !g->cols) return fail(BFS_ERR_OOM, "graph build: CSR arrays");
    g->graph_bytes = sizeof(int64_t) * (size_t)(n + 1) + sizeof(int32_t) * (size_t)(nnz + kColPad);
    const cudaMemcpyKind kind = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    BFS_CUDA_TRY(cudaMemcpyAsync(g->offsets, off, sizeof(int64_t) * (size_t)(n + 1), kind, s));
    if (nnz > 0) BFS_CUDA_TRY(cudaMemcpyAsync(g->cols, cols, sizeof(int32_t) * (size_t)nnz, kind, s));
    k_fill_i32<<<1, 32, 0, s>>>(g->cols + nnz, kColPad, 0);
    BFS_CUDA_TRY(cudaGetLastError());
    Scratch small(&g->mem, s);
    if (!small.get(64)) return fail(BFS_ERR_OOM, "graph build: counters");
    BFS_CUDA_TRY(cudaMemsetAsync(small.p, 0, 64, s));
    int64_t ends[2] = {0, 0};
    BFS_CUDA_TRY(cudaMemcpyAsync(&ends[0], g->offsets, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BFS_CUDA_TRY(cudaMemcpyAsync(&ends[1], g->offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    if (ends[0] != 0 || ends[1] != nnz) return fail(BFS_ERR_INVALID, "row_offsets[0] must be 0 and row_offsets[n] = nnz");
    k_check_csr<<<grid_for(n * 32, 256, g->sm_count), 256, 0, s>>>((const long long*)g->offsets, g->cols, n, nnz,
                                                                 check_symmetry ? 1 : 0, (int*)small.p);
    BFS_CUDA_TRY(cudaGetLastError());
    int bad = 0;
    BFS_CUDA_TRY(cudaMemcpyAsync(&bad, small.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    static const char* why[] = {"", "row offsets decrease or leave [0, nnz]", "a column id lies outside [0, n)",
                                "a row is not strictly ascending (unsorted or duplicate)", "a self-loop",
                                "the CSR is not symmetric"};
    if (bad) return fail(BFS_ERR_INVALID, std::string("invalid CSR: ") + why[bad < 6 ? bad : 0]);
    bfs_status st = build_isolated_bitmap(g, s);
    if (st != BFS_OK) return st;
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    return BFS_OK;
}

}  // namespace bfsrt
