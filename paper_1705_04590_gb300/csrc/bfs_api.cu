// bfs_api.cu -- the extern "C" entry points declared in include/bfs.h.
//
// Argument checking, handle life cycle, the allocator hook, stream ordering
// between runs that share a graph's work buffers, and error reporting
// (status codes + a thread-local message).  All compute is in the kernels of
// bfs_single.cu / bfs_multi.cu / graph_build.cu.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "bfs_internal.h"

namespace bfsrt {

static thread_local std::string t_last_error;

void set_error(const std::string& msg) { t_last_error = msg; }

bfs_status fail(bfs_status st, const std::string& msg) {
    t_last_error = msg;
    return st;
}

bfs_status cuda_fail(cudaError_t e, const char* what) {
    t_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? BFS_ERR_OOM : BFS_ERR_CUDA;
}

void* DeviceAlloc::alloc(size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    if (has_hook && hook.alloc) return hook.alloc(bytes, (void*)s, hook.ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return p;
}

void DeviceAlloc::release(void* p, size_t bytes, cudaStream_t s) {
    if (!p) return;
    if (bytes == 0) bytes = 16;
    if (has_hook && hook.free) {
        hook.free(p, bytes, (void*)s, hook.ctx);
        return;
    }
    cudaFree(p);
}

static void destroy_graph(bfs_graph* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    single_release(g);
    multi_release(g);
    release_dcsc_tiles(g);
    g->mem.release(g->offsets, sizeof(int64_t) * (size_t)(g->n + 1), nullptr);
    g->mem.release(g->cols, sizeof(int32_t) * (size_t)(g->nnz + kColPad), nullptr);
    if (g->cols_hf) g->mem.release(g->cols_hf, sizeof(int32_t) * (size_t)(g->nnz + kColPad), nullptr);
    if (g->bu_heads) g->mem.release(g->bu_heads, sizeof(int32_t) * 8 * (size_t)g->n, nullptr);
    if (g->bu_first) g->mem.release(g->bu_first, sizeof(int32_t) * (size_t)(g->n + 32), nullptr);
    if (g->offsets_in) g->mem.release(g->offsets_in, sizeof(int64_t) * (size_t)(g->n + 1), nullptr);
    if (g->cols_in) g->mem.release(g->cols_in, sizeof(int32_t) * (size_t)(g->nnz + kColPad), nullptr);
    if (g->deg8_in) g->mem.release(g->deg8_in, (size_t)g->n + 32, nullptr);
    if (g->deg8) g->mem.release(g->deg8, (size_t)g->n + 32, nullptr);
    g->mem.release(g->isolated, sizeof(uint32_t) * (size_t)g->W, nullptr);
    if (g->last_done) cudaEventDestroy(g->last_done);
    delete g;
}

static bfs_status new_graph(int64_t n, const bfs_allocator* alloc, bfs_graph** out) {
    if (!out) return fail(BFS_ERR_INVALID, "out handle pointer is NULL");
    *out = nullptr;
    if (n < 1 || n > 2147483647LL) return fail(BFS_ERR_INVALID, "n must lie in [1, 2^31-1]");
    bfs_graph* g = new (std::nothrow) bfs_graph();
    if (!g) return fail(BFS_ERR_OOM, "host allocation of the graph handle");
    g->n = n;
    g->W = (n + 31) / 32;
    if (alloc && alloc->alloc && alloc->free) {
        g->mem.hook = *alloc;
        g->mem.has_hook = true;
    }
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device);
    int coop = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->device);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->last_done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        delete g;
        return cuda_fail(e, "device query");
    }
    if (!coop) {
        destroy_graph(g);
        return fail(BFS_ERR_UNSUPPORTED, "device does not support cooperative launches");
    }
    *out = g;
    return BFS_OK;
}

static bfs_status check_options(const bfs_options* in, bfs_options* out, const bfs_graph* g) {
    bfs_options_default(out);
    if (in) *out = *in;
    if (out->mode < 0 || out->mode > 3) return fail(BFS_ERR_INVALID, "options.mode must be a BFS_MODE_* value");
    if (out->layout != BFS_LAYOUT_CSR && out->layout != BFS_LAYOUT_DCSC_TILED)
        return fail(BFS_ERR_INVALID, "options.layout must be a BFS_LAYOUT_* value");
    if (out->layout == BFS_LAYOUT_DCSC_TILED && !g->dcsc.built)
        return fail(BFS_ERR_UNSUPPORTED, "DCSC layout requested but the graph was built without BFS_FLAG_BUILD_DCSC");
    if (out->alpha < 1 || out->beta < 1) return fail(BFS_ERR_INVALID, "options.alpha and options.beta must be >= 1");
    if (out->parent_mode != BFS_PARENT_ANY && out->parent_mode != BFS_PARENT_MIN_ID)
        return fail(BFS_ERR_INVALID, "options.parent_mode must be a BFS_PARENT_* value");
    if (out->timeout_ms < 0) return fail(BFS_ERR_INVALID, "options.timeout_ms must be >= 0");
    if (out->td_big_degree != 0 && out->td_big_degree < 64) out->td_big_degree = 64;
    if (out->td_chunk != 0 && (out->td_chunk < 64 || out->td_chunk > 4096))
        return fail(BFS_ERR_INVALID, "options.td_chunk must be 0 or lie in [64, 4096]");
    if (out->ctas_per_sm < 0) return fail(BFS_ERR_INVALID, "options.ctas_per_sm must be >= 0");
    if (out->cluster_size != 0 && out->cluster_size != 1 && out->cluster_size != 2 && out->cluster_size != 4 &&
        out->cluster_size != 8 && out->cluster_size != 16)
        return fail(BFS_ERR_INVALID, "options.cluster_size must be 0, 1, 2, 4, 8 or 16");
    if (out->bu_rows != BFS_BU_ROWS_BY_ID && out->bu_rows != BFS_BU_ROWS_HUB_FIRST)
        return fail(BFS_ERR_INVALID, "options.bu_rows must be a BFS_BU_ROWS_* value");
    if (out->bu_rows == BFS_BU_ROWS_HUB_FIRST) {
        if (!g->cols_hf)
            return fail(BFS_ERR_UNSUPPORTED, "hub-first rows requested but the graph was built without "
                                             "BFS_FLAG_BUILD_HUB_FIRST");
        if (out->parent_mode != BFS_PARENT_ANY)
            return fail(BFS_ERR_INVALID, "BFS_BU_ROWS_HUB_FIRST needs BFS_PARENT_ANY (minimum-id parents need id order)");
        if (out->layout != BFS_LAYOUT_CSR) return fail(BFS_ERR_INVALID, "BFS_BU_ROWS_HUB_FIRST needs the CSR layout");
    }
    return BFS_OK;
}

// Order this run after the previous one on the same graph (shared buffers).
static bfs_status order_after_previous(bfs_graph* g, cudaStream_t s) {
    if (g->has_last && g->last_stream != s) BFS_CUDA_TRY(cudaStreamWaitEvent(s, g->last_done, 0));
    return BFS_OK;
}

static bfs_status mark_done(bfs_graph* g, cudaStream_t s) {
    BFS_CUDA_TRY(cudaEventRecord(g->last_done, s));
    g->has_last = true;
    g->last_stream = s;
    return BFS_OK;
}

}  // namespace bfsrt

using namespace bfsrt;

extern "C" {

void bfs_options_default(bfs_options* opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->mode = BFS_MODE_DO;
    opt->layout = BFS_LAYOUT_CSR;
    opt->alpha = 14;
    opt->beta = 24;
    opt->parent_mode = BFS_PARENT_ANY;
    opt->td_big_degree = 0;
    opt->timeout_ms = 10000;
}

bfs_status bfs_graph_create_from_edges(const int32_t* src, const int32_t* dst, int64_t n_edges, int64_t n_vertices,
                                       uint32_t flags, const bfs_allocator* alloc, void* stream, bfs_graph** out) {
    if (out) *out = nullptr;
    if (n_edges < 0) return fail(BFS_ERR_INVALID, "n_edges must be >= 0");
    if (n_edges > 0 && (!src || !dst)) return fail(BFS_ERR_INVALID, "src/dst must not be NULL");
    const bool directed = !(flags & BFS_FLAG_SYMMETRIZE);
    if (directed && (flags & (BFS_FLAG_BUILD_DCSC | BFS_FLAG_BUILD_HUB_FIRST)))
        return fail(BFS_ERR_UNSUPPORTED, "directed graphs: DCSC tiles and hub-first rows are not built");
    bfs_graph* g = nullptr;
    bfs_status st = new_graph(n_vertices, alloc, &g);
    if (st != BFS_OK) return st;
    g->directed = directed;
    cudaStream_t s = (cudaStream_t)stream;
    st = build_csr_from_edges(g, src, dst, n_edges, (flags & BFS_FLAG_DEVICE_PTRS) != 0, s);
    if (st == BFS_OK && (flags & BFS_FLAG_BUILD_DCSC)) st = build_dcsc_tiles(g, s);
    if (st == BFS_OK && (flags & BFS_FLAG_BUILD_HUB_FIRST)) st = build_hub_first_rows(g, s);
    if (st != BFS_OK) {
        std::string msg = bfs_last_error();
        destroy_graph(g);
        set_error(msg);
        return st;
    }
    *out = g;
    return BFS_OK;
}

bfs_status bfs_graph_create_from_edges64(const int64_t* src, const int64_t* dst, int64_t n_edges, int64_t n_vertices,
                                         uint32_t flags, const bfs_allocator* alloc, void* stream, bfs_graph** out) {
    if (out) *out = nullptr;
    if (n_edges < 0) return fail(BFS_ERR_INVALID, "n_edges must be >= 0");
    if (n_edges > 0 && (!src || !dst)) return fail(BFS_ERR_INVALID, "src/dst must not be NULL");
    const bool directed = !(flags & BFS_FLAG_SYMMETRIZE);
    if (directed && (flags & (BFS_FLAG_BUILD_DCSC | BFS_FLAG_BUILD_HUB_FIRST)))
        return fail(BFS_ERR_UNSUPPORTED, "directed graphs: DCSC tiles and hub-first rows are not built");
    bfs_graph* g = nullptr;
    bfs_status st = new_graph(n_vertices, alloc, &g);
    if (st != BFS_OK) return st;
    g->directed = directed;
    cudaStream_t s = (cudaStream_t)stream;
    st = build_csr_from_edges64(g, src, dst, n_edges, (flags & BFS_FLAG_DEVICE_PTRS) != 0, s);
    if (st == BFS_OK && (flags & BFS_FLAG_BUILD_DCSC)) st = build_dcsc_tiles(g, s);
    if (st == BFS_OK && (flags & BFS_FLAG_BUILD_HUB_FIRST)) st = build_hub_first_rows(g, s);
    if (st != BFS_OK) {
        std::string msg = bfs_last_error();
        destroy_graph(g);
        set_error(msg);
        return st;
    }
    *out = g;
    return BFS_OK;
}

bfs_status bfs_graph_create_from_csr(const int64_t* row_offsets, const int32_t* col_ids, int64_t n, int64_t nnz,
                                     uint32_t flags, const bfs_allocator* alloc, void* stream, bfs_graph** out) {
    if (out) *out = nullptr;
    if (!row_offsets) return fail(BFS_ERR_INVALID, "row_offsets must not be NULL");
    if (nnz < 0) return fail(BFS_ERR_INVALID, "nnz must be >= 0");
    if (nnz > 0 && !col_ids) return fail(BFS_ERR_INVALID, "col_ids must not be NULL");
    bfs_graph* g = nullptr;
    bfs_status st = new_graph(n, alloc, &g);
    if (st != BFS_OK) return st;
    g->nnz = nnz;
    cudaStream_t s = (cudaStream_t)stream;
    st = build_csr_from_csr(g, row_offsets, col_ids, (flags & BFS_FLAG_DEVICE_PTRS) != 0,
                            (flags & BFS_FLAG_CHECK_SYMMETRY) != 0, s);
    if (st == BFS_OK && (flags & BFS_FLAG_BUILD_DCSC)) st = build_dcsc_tiles(g, s);
    if (st == BFS_OK && (flags & BFS_FLAG_BUILD_HUB_FIRST)) st = build_hub_first_rows(g, s);
    if (st != BFS_OK) {
        std::string msg = bfs_last_error();
        destroy_graph(g);
        set_error(msg);
        return st;
    }
    *out = g;
    return BFS_OK;
}

bfs_status bfs_graph_info(const bfs_graph* g, int64_t* n, int64_t* nnz, int64_t* device_bytes) {
    if (!g) return fail(BFS_ERR_INVALID, "graph handle is NULL");
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (device_bytes)
        *device_bytes = (int64_t)(g->graph_bytes + g->single.bytes + g->multi.bytes + g->dcsc.bytes);
    return BFS_OK;
}

bfs_status bfs_graph_csr(const bfs_graph* g, const int64_t** row_offsets, const int32_t** col_ids) {
    if (!g) return fail(BFS_ERR_INVALID, "graph handle is NULL");
    if (row_offsets) *row_offsets = g->offsets;
    if (col_ids) *col_ids = g->cols;
    return BFS_OK;
}

bfs_status bfs_graph_copy_csr(const bfs_graph* g, int64_t* offsets_out, int32_t* cols_out, void* stream) {
    if (!g) return fail(BFS_ERR_INVALID, "graph handle is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (offsets_out)
        BFS_CUDA_TRY(cudaMemcpyAsync(offsets_out, g->offsets, sizeof(int64_t) * (size_t)(g->n + 1), cudaMemcpyDefault, s));
    if (cols_out && g->nnz > 0)
        BFS_CUDA_TRY(cudaMemcpyAsync(cols_out, g->cols, sizeof(int32_t) * (size_t)g->nnz, cudaMemcpyDefault, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    return BFS_OK;
}

bfs_status bfs_graph_copy_hub_first(const bfs_graph* g, int32_t* cols_out, void* stream) {
    if (!g || !cols_out) return fail(BFS_ERR_INVALID, "NULL argument");
    if (!g->cols_hf) return fail(BFS_ERR_INVALID, "graph was built without BFS_FLAG_BUILD_HUB_FIRST");
    cudaStream_t s = (cudaStream_t)stream;
    if (g->nnz > 0)
        BFS_CUDA_TRY(cudaMemcpyAsync(cols_out, g->cols_hf, sizeof(int32_t) * (size_t)g->nnz, cudaMemcpyDefault, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    return BFS_OK;
}

bfs_status bfs_graph_copy_row_heads(const bfs_graph* g, int32_t* heads_out, void* stream) {
    if (!g || !heads_out) return fail(BFS_ERR_INVALID, "NULL argument");
    if (!g->bu_heads) return fail(BFS_ERR_INVALID, "graph was built without BFS_FLAG_BUILD_HUB_FIRST");
    cudaStream_t s = (cudaStream_t)stream;
    BFS_CUDA_TRY(cudaMemcpyAsync(heads_out, g->bu_heads, sizeof(int32_t) * 8 * (size_t)g->n, cudaMemcpyDefault, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    return BFS_OK;
}

bfs_status bfs_graph_copy_transpose(const bfs_graph* g, int64_t* offsets_out, int32_t* cols_out, void* stream) {
    if (!g || !offsets_out || !cols_out) return fail(BFS_ERR_INVALID, "NULL argument");
    if (!g->directed) return fail(BFS_ERR_INVALID, "the graph is undirected: its rows are their own transpose");
    cudaStream_t s = (cudaStream_t)stream;
    BFS_CUDA_TRY(cudaMemcpyAsync(offsets_out, g->offsets_in, sizeof(int64_t) * (size_t)(g->n + 1), cudaMemcpyDefault, s));
    if (g->nnz > 0)
        BFS_CUDA_TRY(cudaMemcpyAsync(cols_out, g->cols_in, sizeof(int32_t) * (size_t)g->nnz, cudaMemcpyDefault, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    return BFS_OK;
}

bfs_status bfs_graph_copy_bu_planes(const bfs_graph* g, int32_t* first_out, uint8_t* deg8_out, void* stream) {
    if (!g) return fail(BFS_ERR_INVALID, "NULL graph");
    cudaStream_t s = (cudaStream_t)stream;
    if (first_out) {
        if (!g->bu_first) return fail(BFS_ERR_INVALID, "graph was built without BFS_FLAG_BUILD_HUB_FIRST");
        BFS_CUDA_TRY(cudaMemcpyAsync(first_out, g->bu_first, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDefault, s));
    }
    if (deg8_out) BFS_CUDA_TRY(cudaMemcpyAsync(deg8_out, g->deg8, (size_t)g->n, cudaMemcpyDefault, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    return BFS_OK;
}

bfs_status bfs_graph_dcsc(const bfs_graph* g, bfs_dcsc_layout* out) {
    if (!g || !out) return fail(BFS_ERR_INVALID, "NULL argument");
    if (!g->dcsc.built) return fail(BFS_ERR_INVALID, "graph was built without BFS_FLAG_BUILD_DCSC");
    out->num_blocks = g->dcsc.num_blocks;
    out->reserved = 0;
    out->block_size = g->dcsc.block_size;
    out->tile_ptr = g->dcsc.tile_ptr;
    out->jc = g->dcsc.jc;
    out->cp = g->dcsc.cp;
    out->ir = g->dcsc.ir;
    out->nzc = g->dcsc.nzc;
    return BFS_OK;
}

bfs_status bfs_graph_copy_dcsc(const bfs_graph* g, int64_t* tile_ptr_out, int32_t* jc_out, int64_t* cp_out,
                               int32_t* ir_out, void* stream) {
    if (!g) return fail(BFS_ERR_INVALID, "graph handle is NULL");
    const DcscTiles& D = g->dcsc;
    if (!D.built) return fail(BFS_ERR_INVALID, "graph was built without BFS_FLAG_BUILD_DCSC");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t tiles = (size_t)D.num_blocks * (size_t)D.num_blocks;
    if (tile_ptr_out)
        BFS_CUDA_TRY(cudaMemcpyAsync(tile_ptr_out, D.tile_ptr, sizeof(int64_t) * (tiles + 1), cudaMemcpyDefault, s));
    if (jc_out && D.nzc > 0)
        BFS_CUDA_TRY(cudaMemcpyAsync(jc_out, D.jc, sizeof(int32_t) * (size_t)D.nzc, cudaMemcpyDefault, s));
    if (cp_out) BFS_CUDA_TRY(cudaMemcpyAsync(cp_out, D.cp, sizeof(int64_t) * (size_t)(D.nzc + 1), cudaMemcpyDefault, s));
    if (ir_out && g->nnz > 0)
        BFS_CUDA_TRY(cudaMemcpyAsync(ir_out, D.ir, sizeof(int32_t) * (size_t)g->nnz, cudaMemcpyDefault, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    return BFS_OK;
}

void bfs_graph_destroy(bfs_graph* g) { destroy_graph(g); }

bfs_status bfs_graph_sync(bfs_graph* g, void* stream);

static bfs_status run_common(bfs_graph* g, const int32_t* roots, int32_t k, int32_t* parent_dev, int32_t* level_dev,
                             const bfs_options* opt, void* stream, bfs_stats* stats) {
    if (!g) return fail(BFS_ERR_INVALID, "graph handle is NULL");
    bfs_options o;
    bfs_status st = check_options(opt, &o, g);
    if (st != BFS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->run_mu);
    st = order_after_previous(g, s);
    if (st != BFS_OK) return st;
    st = single_prepare(g, s);
    if (st != BFS_OK) return st;
    st = single_launch(g, roots, k, parent_dev, level_dev, o, s);
    if (st != BFS_OK) return st;
    st = mark_done(g, s);
    if (st != BFS_OK) return st;
    if (stats) return single_collect(g, s, stats);
    return BFS_OK;
}

bfs_status bfs_run(bfs_graph* g, int32_t root, int32_t* parent_dev, int32_t* level_dev, const bfs_options* opt,
                   void* stream, bfs_stats* stats) {
    if (!g) return fail(BFS_ERR_INVALID, "graph handle is NULL");
    if (root < 0 || (int64_t)root >= g->n) return fail(BFS_ERR_INVALID, "root outside [0, n)");
    return run_common(g, &root, 1, parent_dev, level_dev, opt, stream, stats);
}

bfs_status bfs_run_multiroot(bfs_graph* g, const int32_t* roots_host, int32_t k, int32_t* parent_dev,
                             int32_t* level_dev, const bfs_options* opt, void* stream, bfs_stats* stats) {
    if (!g) return fail(BFS_ERR_INVALID, "graph handle is NULL");
    if (!roots_host || k < 1 || (int64_t)k > g->n) return fail(BFS_ERR_INVALID, "need 1 <= k <= n roots");
    std::vector<int32_t> r(roots_host, roots_host + k);
    for (int32_t x : r)
        if (x < 0 || (int64_t)x >= g->n) return fail(BFS_ERR_INVALID, "a root lies outside [0, n)");
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    return run_common(g, r.data(), (int32_t)r.size(), parent_dev, level_dev, opt, stream, stats);
}

bfs_status bfs_run_multi(bfs_graph* g, const int32_t* roots_host, int32_t k, int32_t* level_dev, int32_t* parent_dev,
                         const bfs_options* opt, void* stream) {
    if (!g) return fail(BFS_ERR_INVALID, "graph handle is NULL");
    if (g->directed) return fail(BFS_ERR_UNSUPPORTED, "multi-source search: undirected graphs only");
    if (!roots_host || k < 1) return fail(BFS_ERR_INVALID, "need k >= 1 roots");
    if (!level_dev) return fail(BFS_ERR_INVALID, "level_dev must not be NULL");
    for (int32_t i = 0; i < k; i++)
        if (roots_host[i] < 0 || (int64_t)roots_host[i] >= g->n) return fail(BFS_ERR_INVALID, "a root lies outside [0, n)");
    bfs_options o;
    bfs_status st = check_options(opt, &o, g);
    if (st != BFS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g->run_mu);
    st = order_after_previous(g, s);
    if (st != BFS_OK) return st;
    st = multi_prepare(g, s);
    if (st != BFS_OK) return st;
    st = multi_launch(g, roots_host, k, level_dev, parent_dev, o, s);
    if (st != BFS_OK) return st;
    return mark_done(g, s);
}

bfs_status bfs_autotune(bfs_graph* g, const int32_t* roots_host, int32_t k, const bfs_options* base,
                        bfs_options* best, double* best_ms, void* stream) {
    if (!g || !best) return fail(BFS_ERR_INVALID, "NULL graph or output");
    if (!roots_host || k < 1) return fail(BFS_ERR_INVALID, "need k >= 1 sample roots");
    for (int32_t i = 0; i < k; i++)
        if (roots_host[i] < 0 || (int64_t)roots_host[i] >= g->n) return fail(BFS_ERR_INVALID, "a root lies outside [0, n)");
    bfs_options o0;
    bfs_status st = check_options(base, &o0, g);
    if (st != BFS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // time with both outputs written, as a caller's search would
    const size_t ob = sizeof(int32_t) * (size_t)g->n;
    int32_t* tpar = (int32_t*)g->mem.alloc(ob, s);
    int32_t* tlev = (int32_t*)g->mem.alloc(ob, s);
    if (!tpar || !tlev) {
        g->mem.release(tpar, ob, s);
        g->mem.release(tlev, ob, s);
        return fail(BFS_ERR_OOM, "autotune: output buffers");
    }
    static const int alphas[] = {6, 14, 24, 32, 96};
    static const int betas[] = {12, 24, 64, 128};
    static const int bigs[] = {64, 96, 256};
    static const int chunks[] = {128, 256, 512, 1024};
    static const int ctas[] = {1, 0};   // 1 CTA per SM, or as many as fit
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BFS_CUDA_TRY(cudaEventCreate(&e0));
    BFS_CUDA_TRY(cudaEventCreate(&e1));
    double best_t = -1.0;
    bfs_options win = o0;
    // mean ms per search of `o` over the sample roots (one warm-up search first)
    auto trial = [&](const bfs_options& o) -> double {
        st = run_common(g, roots_host, 1, tpar, tlev, &o, stream, nullptr);
        if (st != BFS_OK) return -1.0;
        if (cudaEventRecord(e0, s) != cudaSuccess) { st = BFS_ERR_CUDA; return -1.0; }
        for (int32_t i = 0; i < k && st == BFS_OK; i++) st = run_common(g, roots_host + i, 1, tpar, tlev, &o, stream, nullptr);
        if (st != BFS_OK) return -1.0;
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            st = BFS_ERR_CUDA;
            return -1.0;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms / k;
    };
    auto consider = [&](const bfs_options& o) {
        const double per = trial(o);
        if (per >= 0 && (best_t < 0 || per < best_t)) {
            best_t = per;
            win = o;
        }
    };
    // the direction thresholds and the hub cut-off on a grid, then the launch knobs one at a time
    for (int a : alphas)
        for (int b : betas)
            for (int big : bigs) {
                if (st != BFS_OK) break;
                bfs_options o = o0;
                o.mode = BFS_MODE_DO;
                o.alpha = a;
                o.beta = b;
                o.td_big_degree = big;
                consider(o);
            }
    const bfs_options grid_win = win;
    for (int c : chunks) {
        if (st != BFS_OK) break;
        bfs_options o = grid_win;
        o.td_chunk = c;
        consider(o);
    }
    const bfs_options chunk_win = win;
    for (int c : ctas) {
        if (st != BFS_OK) break;
        bfs_options o = chunk_win;
        o.ctas_per_sm = c;
        consider(o);
    }
    // cluster levels (CSR searches of undirected graphs): off, clusters of 8, of 16
    if (!g->directed && o0.layout == BFS_LAYOUT_CSR) {
        static const int clus[] = {1, 8, 16};
        const bfs_options ctas_win = win;
        for (int c : clus) {
            if (st != BFS_OK) break;
            bfs_options o = ctas_win;
            o.cluster_size = c;
            consider(o);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    g->mem.release(tpar, ob, s);
    g->mem.release(tlev, ob, s);
    if (st != BFS_OK) return st;
    st = bfs_graph_sync(g, stream);
    if (st != BFS_OK) return st;
    *best = win;
    if (best_ms) *best_ms = best_t;
    return BFS_OK;
}

bfs_status bfs_debug_set_barrier_extra(bfs_graph* g, int32_t extra) {
    if (!g) return fail(BFS_ERR_INVALID, "graph handle is NULL");
    if (extra < 0) return fail(BFS_ERR_INVALID, "extra must be >= 0");
    std::lock_guard<std::mutex> lk(g->run_mu);
    g->debug_barrier_extra = extra;
    return BFS_OK;
}

bfs_status bfs_graph_sync(bfs_graph* g, void* stream) {
    if (!g) return fail(BFS_ERR_INVALID, "graph handle is NULL");
    std::lock_guard<std::mutex> lk(g->run_mu);
    cudaStream_t s = (cudaStream_t)stream;
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    if (g->last_done) BFS_CUDA_TRY(cudaEventSynchronize(g->last_done));
    if (g->single.ready) {
        bfs_status st = single_collect(g, s, nullptr);
        if (st != BFS_OK) return st;
    }
    if (g->multi.ready) return multi_collect_status(g, s);
    return BFS_OK;
}

const char* bfs_status_string(bfs_status st) {
    switch (st) {
        case BFS_OK: return "BFS_OK";
        case BFS_ERR_INVALID: return "BFS_ERR_INVALID";
        case BFS_ERR_OOM: return "BFS_ERR_OOM";
        case BFS_ERR_CUDA: return "BFS_ERR_CUDA";
        case BFS_ERR_TIMEOUT: return "BFS_ERR_TIMEOUT";
        case BFS_ERR_BUSY: return "BFS_ERR_BUSY";
        case BFS_ERR_NOT_READY: return "BFS_ERR_NOT_READY";
        case BFS_ERR_UNSUPPORTED: return "BFS_ERR_UNSUPPORTED";
    }
    return "BFS_ERR_UNKNOWN";
}

const char* bfs_last_error(void) { return t_last_error.c_str(); }

const char* bfs_version(void) { return "gb300-dobfs 0.1 (sm_103a)"; }

}  // extern "C"
