// bfs_internal.h -- host-side structures shared by the library's translation
// units (not part of the public ABI; see include/bfs.h for that).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>

#include "../../include/bfs.h"

namespace bfsrt {

// thread-local last error message + helpers (bfs_api.cpp)
void set_error(const std::string& msg);
bfs_status fail(bfs_status st, const std::string& msg);
bfs_status cuda_fail(cudaError_t e, const char* what);

#define BFS_CUDA_TRY(expr)                                     \
    do {                                                       \
        cudaError_t e__ = (expr);                              \
        if (e__ != cudaSuccess) return bfsrt::cuda_fail(e__, #expr); \
    } while (0)

// Device memory through the user hook or cudaMalloc.
struct DeviceAlloc {
    bfs_allocator hook{};
    bool has_hook = false;
    void* alloc(size_t bytes, cudaStream_t s);
    void release(void* p, size_t bytes, cudaStream_t s);
};

// Per-graph buffers of the single-source search, reused by every run.
struct SingleWork {
    DeviceAlloc* mem = nullptr;    // allocator of these buffers (null: the graph's)
    bool ready = false;
    unsigned* visited = nullptr;   // [W]
    unsigned* front0 = nullptr;    // [W]
    unsigned* front1 = nullptr;    // [W]
    int* queue0 = nullptr;         // [n]
    int* queue1 = nullptr;         // [n]
    unsigned char* lv8 = nullptr;  // [W * 32] staged levels (one byte per vertex, whole words)
    unsigned* pfirst = nullptr;    // [W] bit v: v's parent is its first hub-first neighbour (bu_first[v])
    int* level_scratch = nullptr;  // [n] levels for MIN_ID parents when the caller wants none (lazy)
    void* tasks = nullptr;         // top-down edge-chunk descriptors
    long long task_cap = 0;
    void* ctrl = nullptr;          // bfsk::Ctrl
    bfs_level_record* records = nullptr;  // [rec_cap] device
    int rec_cap = 0;
    int* roots_dev = nullptr;      // [n] staging for multi-root seeds
    int* roots_pinned = nullptr;   // host pinned staging
    long long roots_cap = 0;
    size_t bytes = 0;
    int grid = 0, block = 0;       // cooperative launch shape
    int clu_grid[5] = {0, 0, 0, 0, 0};   // co-resident CTAs of a launch in clusters of 1, 2, 4, 8, 16 (0 = not asked yet)
};

// Buffers of one multi-source (64-lane) search state: bfs_run_multi's own,
// and one per graph slot of a server.
struct MultiWork {
    DeviceAlloc* mem = nullptr;    // allocator of these buffers (null: the graph's)
    bool ready = false;
    unsigned long long* seen = nullptr;   // [n] lane masks
    unsigned long long* front = nullptr;  // [n]
    unsigned long long* next = nullptr;   // [n]
    void* ctrl = nullptr;                 // bfsk::MCtrl
    void* tasks = nullptr;                // bfsk::MTask[task_cap]
    void* hubmask = nullptr;              // uint64[task_cap] lane masks of chunked rows
    long long task_cap = 0;
    void* lanes = nullptr;                // bfsk::LaneTable
    int* q0 = nullptr;                    // [n+64] vertex queues (frontier / touched)
    int* q1 = nullptr;
    size_t bytes = 0;
    int grid = 0, block = 0;
};

struct DcscTiles {
    bool built = false;
    int num_blocks = 0;            // p
    long long block_size = 0;      // B (multiple of 32)
    int bits = 0;                  // bits of B
    int64_t* tile_ptr = nullptr;   // [p*p+1]
    int32_t* jc = nullptr;         // [nzc] column within block
    int64_t* cp = nullptr;         // [nzc+1] IR position of each column
    int32_t* ir = nullptr;         // [nnz + kColPad] row within block
    long long nzc = 0;
    size_t bytes = 0;
};

}  // namespace bfsrt

struct bfs_graph {
    int64_t n = 0;
    int64_t nnz = 0;
    int device = 0;
    int64_t* offsets = nullptr;     // [n+1]
    int32_t* cols = nullptr;        // [nnz + kColPad]
    uint32_t* isolated = nullptr;   // [W] bit v set when deg(v) = 0 or v >= n
    int32_t* cols_hf = nullptr;     // [nnz + kColPad] rows ordered by neighbour degree (BFS_FLAG_BUILD_HUB_FIRST)
    // [8n] heads of the hub-first rows, one 32-byte record per vertex:
    // [8u..8u+7] = {deg(u), r0 .. r6} with r the row's first ids (0 past its end)
    int32_t* bu_heads = nullptr;
    // [n + 32] first id of each hub-first row (0 for degree 0), built with the heads
    int32_t* bu_first = nullptr;
    uint8_t* deg8 = nullptr;        // [n + 32] min(deg(v), 255) (out-degree of a directed graph)
    // a directed graph: offsets/cols hold the out-edge rows (top-down), these the
    // transpose (the in-edge rows a bottom-up step scans); null when undirected
    bool directed = false;
    int64_t* offsets_in = nullptr;  // [n+1]
    int32_t* cols_in = nullptr;     // [nnz + kColPad]
    uint8_t* deg8_in = nullptr;     // [n + 32] min(in-degree, 255)
    int64_t W = 0;                  // bitmap words
    int64_t n_active = 0;           // vertices with degree > 0
    int64_t max_degree = 0;         // largest degree (largest in- or out-degree of a directed graph)
    int32_t debug_barrier_extra = 0;   // testing: arrivals every grid barrier waits for in vain
    size_t graph_bytes = 0;
    bfsrt::DeviceAlloc mem;
    bfsrt::SingleWork single;
    bfsrt::MultiWork multi;
    bfsrt::DcscTiles dcsc;
    std::mutex run_mu;              // serialises runs on the shared work buffers
    cudaEvent_t last_done = nullptr;   // completion of the last enqueued run
    cudaStream_t last_stream = nullptr;
    bool has_last = false;
    unsigned run_counter = 0;
    int sm_count = 0;
};

namespace bfsrt {

// the allocator a work-buffer set draws from: its own (a server's) or the graph's
template <typename Work>
inline DeviceAlloc& mem_of(bfs_graph* g, Work& w) {
    return w.mem ? *w.mem : g->mem;
}

constexpr int64_t kColPad = 32;  // readable slack after col_ids (vector loads past the last row)

// graph_build.cu
bfs_status build_csr_from_edges(bfs_graph* g, const int32_t* src, const int32_t* dst, int64_t m,
                                bool device_ptrs, cudaStream_t s);
bfs_status build_csr_from_csr(bfs_graph* g, const int64_t* off, const int32_t* cols, bool device_ptrs,
                              bool check_symmetry, cudaStream_t s);
bfs_status build_csr_from_edges64(bfs_graph* g, const int64_t* src, const int64_t* dst, int64_t m, bool device_ptrs,
                                  cudaStream_t s);
bfs_status build_isolated_bitmap(bfs_graph* g, cudaStream_t s);
bfs_status build_dcsc_tiles(bfs_graph* g, cudaStream_t s);
bfs_status build_hub_first_rows(bfs_graph* g, cudaStream_t s);   // hub_first.cu
void release_dcsc_tiles(bfs_graph* g);

// bfs_single.cu
bfs_status single_prepare(bfs_graph* g, cudaStream_t s);
bfs_status single_launch(bfs_graph* g, const int32_t* roots_host, int32_t k, int32_t* parent,
                         int32_t* level, const bfs_options& opt, cudaStream_t s);
bfs_status single_collect(bfs_graph* g, cudaStream_t s, bfs_stats* stats);
void single_release(bfs_graph* g);
// the same on a caller-held search state (the server's concurrent searches)
bfs_status single_prepare_work(bfs_graph* g, SingleWork& w, cudaStream_t s, int grid);
bfs_status single_launch_work(bfs_graph* g, SingleWork& w, const int32_t* roots_host, int32_t k, int32_t* parent,
                              int32_t* level, const bfs_options& opt, cudaStream_t s);
void single_release_work(bfs_graph* g, SingleWork& w);
size_t single_ctrl_bytes();
unsigned single_ctrl_status(const void* ctrl_host);

// bfs_multi.cu
bfs_status multi_prepare(bfs_graph* g, cudaStream_t s);
bfs_status multi_launch(bfs_graph* g, const int32_t* roots_host, int32_t k, int32_t* level,
                        int32_t* parent, const bfs_options& opt, cudaStream_t s);
bfs_status multi_collect_status(bfs_graph* g, cudaStream_t s);
void multi_release(bfs_graph* g);
bfs_status multi_alloc(bfs_graph* g, MultiWork& w, cudaStream_t s);
void multi_free(bfs_graph* g, MultiWork& w);

// Server driver (bfs_multi.cu): one persistent launch per step of a slot.
size_t ms_lane_table_bytes();
void ms_lane_table_set(void* table_host, int lane, int32_t* row, int start, int root);
int ms_serve_max_grid(bfs_graph* g, MultiWork& w);
bfs_status ms_serve_reset(bfs_graph* g, MultiWork& w, cudaStream_t s);
// Admit `newmask` lanes (lane table copied from lane_table_host), clear the
// stale bits of `drop` lanes, then run up to max_iters levels of `active`
// lanes from iteration iter0 on `grid` CTAs; the slot's control block is
// copied to ctrl_pinned (host, pinned) when the launch ends.
bfs_status ms_serve_launch(bfs_graph* g, MultiWork& w, const void* lane_table_host, unsigned long long newmask,
                           unsigned long long drop, unsigned long long active, int iter0, int max_iters, int grid,
                           void* ctrl_pinned, cudaStream_t s);

}  // namespace bfsrt
