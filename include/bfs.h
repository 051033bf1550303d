/*
 * bfs.h -- C ABI of a single-GPU direction-optimizing breadth-first search
 * library for GB300 (sm_103a).
 *
 * The operations follow Bulu\c{c}, Beamer, Madduri, Asanovic, Patterson,
 * "Distributed-Memory Breadth-First Search on Massive Graphs" (2015):
 *   - the problem statement of Algorithm 1/2: input G(V, E) and a source s;
 *     output parent[v] = the parent of v in a breadth-first spanning tree,
 *     -1 if v is unreachable, parent[s] = s; the parent of a vertex d hops
 *     from s is any vertex d-1 hops from s with an edge to it ("Breadth-First
 *     Search");
 *   - top-down steps (Algorithm 1), bottom-up steps (Algorithm 2) and the
 *     per-level choice between them ("Parallel Direction-Optimizing BFS");
 *   - CSR storage, or DCSC for hypersparse sub-matrices ("Graph
 *     Representation"); graphs are undirected, duplicates and self-loops are
 *     pruned ("Data Sets").
 *
 * Conventions for every call:
 *   - Every function returns a bfs_status; no C++ exception crosses the ABI.
 *     On error a message is available from bfs_last_error() (thread-local,
 *     valid until the next call on that thread).
 *   - Vertex ids are int32_t (n <= 2^31 - 1); edge counts and offsets are
 *     int64_t.
 *   - "stream" is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued on it; outputs are valid once the stream has
 *     reached the point of the call (unless a function says it synchronises).
 *   - The library owns graph storage and per-graph work buffers (allocated
 *     through the bfs_allocator given at creation, or cudaMalloc if NULL).  The
 *     caller owns every output buffer and every stream.
 *   - A failed call leaves no partially built object behind.
 */
#ifndef BFS_GB300_H
#define BFS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BFS_OK = 0,
    BFS_ERR_INVALID = 1,     /* bad argument (NULL handle, root out of range, bad sizes, bad CSR) */
    BFS_ERR_OOM = 2,         /* device or host allocation failed */
    BFS_ERR_CUDA = 3,        /* a CUDA runtime call failed (message names it) */
    BFS_ERR_TIMEOUT = 4,     /* a bounded device wait (grid barrier) ran out; outputs undefined */
    BFS_ERR_BUSY = 5,        /* server: no free capacity (queue full) */
    BFS_ERR_NOT_READY = 6,   /* server: ticket still in flight */
    BFS_ERR_UNSUPPORTED = 7  /* option or layout not supported for this graph/device */
} bfs_status;

typedef struct bfs_graph bfs_graph;
typedef struct bfs_server bfs_server;

/*
 * Device memory hook.  alloc(bytes, stream, ctx) returns device memory (NULL
 * on failure); free(ptr, bytes, stream, ctx) releases it.  Memory may be
 * stream-ordered on `stream`.  NULL hook => cudaMalloc / cudaFree.
 */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
    void* ctx;
} bfs_allocator;

/* graph construction flags */
#define BFS_FLAG_DEVICE_PTRS   1u  /* input arrays are device pointers (else host memory) */
#define BFS_FLAG_SYMMETRIZE    2u  /* store each edge in both rows (undirected); required for edge lists */
#define BFS_FLAG_BUILD_DCSC    4u  /* also build the column-block DCSC tiles (layout BFS_LAYOUT_DCSC_TILED) */
#define BFS_FLAG_CHECK_SYMMETRY 8u /* from_csr: verify that the CSR is symmetric (one extra pass) */
#define BFS_FLAG_BUILD_HUB_FIRST 16u /* also store a copy of every row ordered by neighbour degree, highest
                                        first, ties by id (bottom-up option BFS_BU_ROWS_HUB_FIRST), and
                                        per vertex a 32-byte head (its degree and the first 7 ids of
                                        that row): 4*nnz + 32*n more device bytes */

/* search direction policy ("Parallel Direction-Optimizing BFS") */
#define BFS_MODE_DO       0   /* per level: top-down or bottom-up by the alpha/beta rule */
#define BFS_MODE_TD_ONLY  1   /* every level top-down (Algorithm 1) */
#define BFS_MODE_BU_ONLY  2   /* every level bottom-up (Algorithm 2) */
#define BFS_MODE_RANDOM   3   /* per level a seeded coin flip (testing: levels must not change) */

#define BFS_LAYOUT_CSR          0
#define BFS_LAYOUT_DCSC_TILED   1

#define BFS_PARENT_ANY     0  /* any valid parent (whichever claim wins) */
#define BFS_PARENT_MIN_ID  1  /* the minimum-id valid parent: the (select2nd, min) semiring */

/*
 * Options of one search; pass NULL for the defaults (DO, CSR, alpha 14,
 * beta 24, ANY parent, 10 s barrier limit).  Direction rule, at the start of
 * level d with frontier size n_f, frontier degree sum m_f and degree sum m_u
 * of the vertices not yet reached: in top-down, switch to bottom-up when
 * m_f * alpha > m_u; in bottom-up, switch to top-down when n_f * beta < n.
 * Levels never depend on these choices, only the work does.
 */
typedef struct {
    int32_t mode;          /* BFS_MODE_* */
    int32_t layout;        /* BFS_LAYOUT_*; DCSC needs a graph built with BFS_FLAG_BUILD_DCSC */
    int32_t alpha;         /* >= 1 */
    int32_t beta;          /* >= 1 */
    int32_t parent_mode;   /* BFS_PARENT_* */
    int32_t td_big_degree; /* top-down: frontier vertices above this degree are split into edge chunks
                              shared by all warps (0 = tuned default) */
    int64_t timeout_ms;    /* limit of every device-side wait; 0 = default 10000 */
    uint64_t seed;         /* BFS_MODE_RANDOM only */
    int32_t bu_rows;       /* order in which bottom-up steps scan a row: BFS_BU_ROWS_BY_ID (stored order,
                              the paper's) or BFS_BU_ROWS_HUB_FIRST (needs BFS_FLAG_BUILD_HUB_FIRST, the
                              CSR layout and BFS_PARENT_ANY).  Levels are the same; the bottom-up
                              examination counts and the parents chosen follow the order */
    int32_t td_chunk;      /* top-down: edges per chunk task of a vertex above td_big_degree, 64..4096
                              (0 = tuned default 128) */
    int32_t ctas_per_sm;   /* CTAs per SM of the persistent single-source launch, 1 .. the resident
                              maximum (0 = the maximum); fewer means fewer arrivals per grid barrier */
    int32_t cluster_size;  /* CSR single-source searches of an undirected graph: CTAs per thread-block
                              cluster (2, 4, 8 or 16), whose first cluster runs top-down levels with
                              a small frontier alone (frontier in distributed shared memory, one
                              hardware cluster barrier per level) while the rest of the grid waits;
                              1 = off; 0 = automatic (16 on graphs of maximum degree <= 32, where
                              the levels are many and small, else off).  A cluster launch may hold
                              fewer CTAs than the plain one.  Ignored by DCSC, directed graphs and
                              the allocation-free entry point */
} bfs_options;

#define BFS_BU_ROWS_BY_ID     0
#define BFS_BU_ROWS_HUB_FIRST 1

void bfs_options_default(bfs_options* opt);

/* One record per level of a search (device counters copied back). */
typedef struct {
    int32_t dir;          /* 0 top-down, 1 bottom-up */
    int32_t misses;       /* bottom-up over the hub-first rows: searchers whose first neighbour was not
                             in the frontier and that have more neighbours (0 otherwise) */
    int64_t nf;           /* frontier size at the start of the level */
    int64_t mf;           /* sum of degrees over the frontier */
    int64_t nnext;        /* vertices discovered by the level */
    int64_t mnext;        /* their degree sum */
    int64_t scanned;      /* bottom-up: unvisited vertices with degree > 0 that searched */
    int64_t examined;     /* top-down: m_f; bottom-up: sum over searching vertices of the 1-based
                             position of the first frontier neighbour in sorted order, or the degree */
    int64_t t_ns;         /* device time from the end of initialisation to the end of this level */
    int64_t aux;          /* top-down: edge-chunk tasks, or -1 for a level thread-block cluster 0 ran
                             alone (options.cluster_size); bottom-up: searchers continued past their
                             first window (id-ordered rows) or row head (hub-first rows): the long list */
    int64_t t_mid_ns;     /* device time at the level's first internal barrier (0 if none) */
} bfs_level_record;

typedef struct {
    int32_t num_levels;        /* levels with a non-empty frontier */
    int32_t levels_capacity;   /* in: entries available at `levels` (may be 0) */
    bfs_level_record* levels;  /* in: host array or NULL; out: min(num_levels, capacity) records */
    int64_t vertices_reached;
    int64_t edges_examined;    /* sum of `examined` over all levels */
    int64_t t_init_ns;         /* device time of the initialisation (output staging, bitmaps, root) */
    int64_t t_final_ns;        /* device time from the end of the last level to the last CTA's end of the
                                  final pass that writes level[] and parent[] (0 when none ran) */
} bfs_stats;

/* ----------------------------------------------------------------- graphs */

/*
 * Build a graph from an edge list (src[i], dst[i]), i < n_edges, ids in
 * [0, n_vertices).  Self-loops and duplicate edges are dropped and each row is
 * sorted ascending ("Graph Representation", "Data Sets").  With
 * BFS_FLAG_SYMMETRIZE the graph is undirected (each edge in both rows).
 * Without it the graph is directed ("Data Sets": the algorithms apply to
 * directed graphs): edge i runs src[i] -> dst[i]; the library stores the
 * out-edge rows (top-down steps expand them) and their transpose (the in-edge
 * rows bottom-up steps scan: "Data Decomposition"), 8*nnz + 8*n more device
 * bytes; a search follows edge directions; BFS_FLAG_BUILD_DCSC and
 * BFS_FLAG_BUILD_HUB_FIRST are refused (UNSUPPORTED), and so are
 * bfs_run_multi and the server on such a graph.  With
 * BFS_FLAG_DEVICE_PTRS, src/dst are device pointers, else host pointers
 * (copied in chunks).  The build runs on `stream` and returns when the graph
 * is ready.  Isolated vertices keep their ids.  *out receives the handle.
 * Errors: INVALID (NULL pointers, n_vertices outside [1, 2^31-1], an id out of
 * range, no SYMMETRIZE flag), OOM, CUDA.
 */
bfs_status bfs_graph_create_from_edges(const int32_t* src, const int32_t* dst, int64_t n_edges,
                                       int64_t n_vertices, uint32_t flags, const bfs_allocator* alloc,
                                       void* stream, bfs_graph** out);

/*
 * The same with 64-bit endpoint arrays (the paper stores 64-bit vertex ids):
 * src[i], dst[i] must lie in [0, n_vertices), n_vertices <= 2^31 - 1 (ids are
 * int32 on the device).  The arrays are narrowed to int32 in chunks (on the
 * host, or with BFS_FLAG_DEVICE_PTRS on the device after a range check);
 * an id out of range gives INVALID.  Otherwise as above.
 */
bfs_status bfs_graph_create_from_edges64(const int64_t* src, const int64_t* dst, int64_t n_edges,
                                         int64_t n_vertices, uint32_t flags, const bfs_allocator* alloc,
                                         void* stream, bfs_graph** out);

/*
 * Build a graph from a CSR that is already undirected: row_offsets[n+1]
 * (int64, row_offsets[0] = 0, non-decreasing), col_ids[nnz] (int32, each row
 * strictly ascending, no self-loops).  The arrays are copied.  The row rules
 * and id ranges are checked on the device (INVALID if broken); symmetry only
 * with BFS_FLAG_CHECK_SYMMETRY.
 */
bfs_status bfs_graph_create_from_csr(const int64_t* row_offsets, const int32_t* col_ids, int64_t n,
                                     int64_t nnz, uint32_t flags, const bfs_allocator* alloc, void* stream,
                                     bfs_graph** out);

/* n, nnz (directed entries = 2 x undirected edges) and device bytes held; any pointer may be NULL. */
bfs_status bfs_graph_info(const bfs_graph* g, int64_t* n, int64_t* nnz, int64_t* device_bytes);

/*
 * Device pointers of the stored CSR (row_offsets int64[n+1], col_ids
 * int32[nnz]); owned by the graph, valid until bfs_graph_destroy.
 */
bfs_status bfs_graph_csr(const bfs_graph* g, const int64_t** row_offsets, const int32_t** col_ids);

/*
 * Copy the stored CSR into caller buffers (host or device; the copy kind is
 * inferred): offsets_out int64[n+1], cols_out int32[nnz] (either may be
 * NULL).  Synchronises `stream`.
 */
bfs_status bfs_graph_copy_csr(const bfs_graph* g, int64_t* offsets_out, int32_t* cols_out, void* stream);

/*
 * Copy the hub-first column ids (BFS_FLAG_BUILD_HUB_FIRST) into caller memory
 * (host or device, int32[nnz]): row u holds the same neighbours as the CSR's
 * row u, ordered by neighbour degree, highest first, ties by id ascending;
 * row bounds are the CSR offsets.  Synchronises `stream`.  Errors: INVALID
 * (NULL argument, graph built without the flag), CUDA.
 */
bfs_status bfs_graph_copy_hub_first(const bfs_graph* g, int32_t* cols_out, void* stream);

/*
 * Copy the row heads that BFS_FLAG_BUILD_HUB_FIRST stores beside the hub-first
 * rows into caller memory (host or device, int32[8n]): record u is
 * heads_out[8u .. 8u+7] = {deg(u), r0, .., r6}, where r0.. are the first
 * min(deg(u), 7) ids of u's hub-first row and the rest 0.  Bottom-up steps
 * over the hub-first rows (Algorithm 2 in that order) probe these ids first.
 * Synchronises `stream`.  Errors: INVALID (NULL argument, graph built without
 * the flag), CUDA.
 */
bfs_status bfs_graph_copy_row_heads(const bfs_graph* g, int32_t* heads_out, void* stream);

/*
 * Copy two per-vertex planes into caller memory (host or device); either
 * pointer may be NULL to skip it.
 *   first_out (int32[n], needs BFS_FLAG_BUILD_HUB_FIRST): bits 0-30 the first
 *     id of each vertex's hub-first row, bit 31 set when the vertex has two or
 *     more neighbours; 0 for a vertex of degree 0.  Algorithm 2 probes this
 *     neighbour first (on R-MAT graphs it is the hit for most searchers), and a
 *     bottom-up sweep streams this plane in vertex order.
 *   deg8_out (uint8[n], every graph): min(deg(v), 255), read by top-down steps
 *     for the degree sum of the next frontier.
 * Synchronises `stream`.  Errors: INVALID (NULL graph, first_out on a graph
 * built without the flag), CUDA.
 */
bfs_status bfs_graph_copy_bu_planes(const bfs_graph* g, int32_t* first_out, uint8_t* deg8_out, void* stream);

/*
 * A directed graph's transpose (the in-edge rows) into caller memory (host or
 * device): offsets_out int64[n+1], cols_out int32[nnz]; row v holds the sorted
 * sources of the edges into v.  Synchronises `stream`.  Errors: INVALID (NULL
 * argument, undirected graph), CUDA.
 */
bfs_status bfs_graph_copy_transpose(const bfs_graph* g, int64_t* offsets_out, int32_t* cols_out, void* stream);

/*
 * Device pointers of the DCSC tiles built with BFS_FLAG_BUILD_DCSC ("Graph
 * Representation": IR row ids, JC ids of non-empty columns, CP column
 * pointers).  Vertices are cut into num_blocks blocks of block_size
 * consecutive ids; tile (i, j) holds entries with row in block i and column
 * in block j, stored i-major as DCSC over its columns:
 *   tile_ptr[i*p + j] .. tile_ptr[i*p + j + 1]   range of JC/CP entries
 *   jc[x]       column - j*block_size, ascending within the tile
 *   cp[x] .. cp[x+1]   range of ir entries of that column
 *   ir[e]       row - i*block_size, ascending within a column
 * Owned by the graph; valid until bfs_graph_destroy.  INVALID if not built.
 */
typedef struct {
    int32_t num_blocks;          /* p */
    int32_t reserved;
    int64_t block_size;          /* vertices per block (multiple of 32) */
    const int64_t* tile_ptr;     /* [p*p + 1] */
    const int32_t* jc;           /* [nzc] */
    const int64_t* cp;           /* [nzc + 1] */
    const int32_t* ir;           /* [nnz] */
    int64_t nzc;                 /* non-empty (tile, column) pairs */
} bfs_dcsc_layout;
bfs_status bfs_graph_dcsc(const bfs_graph* g, bfs_dcsc_layout* out);

/*
 * Copy the DCSC tile arrays into caller buffers (host or device; sizes from
 * bfs_graph_dcsc: tile_ptr p*p+1, jc nzc, cp nzc+1, ir nnz).  Any pointer may
 * be NULL.  Synchronises `stream`.  INVALID if the tiles were not built.
 */
bfs_status bfs_graph_copy_dcsc(const bfs_graph* g, int64_t* tile_ptr_out, int32_t* jc_out, int64_t* cp_out,
                               int32_t* ir_out, void* stream);

void bfs_graph_destroy(bfs_graph* g);

/* ----------------------------------------------------------------- search */

/*
 * Breadth-first search from `root` (Algorithm 1/2 with the per-level
 * direction choice).  parent_dev / level_dev: caller-owned device arrays of n
 * int32, either may be NULL.  level[v] = hop distance or -1; parent as in the
 * problem statement.  Levels are exact; parents are any valid parent (or the
 * minimum one with BFS_PARENT_MIN_ID).  A degree-0 root is valid (only it is
 * reached).  The whole level loop runs on the device in one launch (no host
 * round trip per level).  Asynchronous on `stream`, unless stats != NULL: then
 * the call synchronises the stream and fills *stats, and a device-side
 * timeout is reported as BFS_ERR_TIMEOUT.  Without stats, a timeout is
 * reported by the next call that synchronises on this graph
 * (bfs_graph_sync).  Runs on one graph handle are serialised by the library
 * (they share work buffers).  Errors: INVALID (root outside [0, n), bad
 * options), UNSUPPORTED, CUDA, TIMEOUT.
 */
bfs_status bfs_run(bfs_graph* g, int32_t root, int32_t* parent_dev, int32_t* level_dev,
                   const bfs_options* opt, void* stream, bfs_stats* stats);

/*
 * One search from a set of roots, all at level 0 (level = distance to the
 * nearest root; parent[r] = r for each root).  For a disjoint union of graphs
 * with one root per part this is each part's own BFS, which is how an uneven
 * batch of many graphs runs in one launch.  roots_host: k distinct ids
 * (repeats are ignored), 1 <= k <= n.  Otherwise as bfs_run.
 */
bfs_status bfs_run_multiroot(bfs_graph* g, const int32_t* roots_host, int32_t k, int32_t* parent_dev,
                             int32_t* level_dev, const bfs_options* opt, void* stream, bfs_stats* stats);

/*
 * Batched multi-source BFS: k independent searches (roots_host[0..k-1],
 * repeats allowed), packed 64 at a time as per-vertex 64-bit lane masks and
 * advanced together, one fused persistent launch per 64 roots.
 * level_dev: device int32[k][n] row-major (row i = search from roots_host[i]).
 * parent_dev: NULL, or int32[k][n]: for each reached v != root the minimum-id
 * neighbour one level closer (BFS_PARENT_MIN_ID semantics).  Asynchronous
 * on `stream`.  Errors: INVALID, OOM, CUDA.
 */
bfs_status bfs_run_multi(bfs_graph* g, const int32_t* roots_host, int32_t k, int32_t* level_dev,
                         int32_t* parent_dev, const bfs_options* opt, void* stream);

/*
 * Allocation-free search for callers that cannot allocate device memory: a
 * caller whose device memory is fully pre-allocated by its own pool or arena,
 * or one on a path where cudaMalloc/cudaFree -- which may synchronise the
 * device and take time that cannot be bounded -- must not run.  The paper has
 * no counterpart; this is the direction-optimizing search of bfs_run with
 * default options over a caller-provided CSR, with every work buffer in one
 * fixed device array of about 14 MB compiled into the library.
 *   row_offsets: device int64[n+1], 8-byte aligned; col_ids: device
 *   int32[nnz], 16-byte aligned, holding an undirected graph as
 *   bfs_graph_create_from_csr accepts it (rows strictly ascending, no
 *   self-loops, symmetric), readable for 32 entries past nnz (16-byte loads
 *   may run up to 28 bytes beyond the last row; those values are ignored).
 *   parent_dev / level_dev: device int32[n], 4-byte aligned, either may be
 *   NULL.  Limits: 1 <= n <= 1,048,576 and nnz <= 16,777,216, else
 *   BFS_ERR_INVALID with a message naming the limit; a misaligned pointer
 *   also gives BFS_ERR_INVALID (checked on the host, nothing is launched).
 * Calls no cudaMalloc, cudaFree or allocating routine.  The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress, once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call shares the array: calls whose work overlaps on the GPU
 * (on different streams) race and must be ordered by the caller.  Each call
 * re-initialises all of it that it reads.  Asynchronous on `stream`; no device
 * error is reported back: a search whose grid-barrier wait ran out of time
 * (10 s) leaves parent/level partly written with no status.  A caller that
 * needs to know must check the outputs itself (level[root] == 0, and every
 * reached v has level[parent[v]] == level[v] - 1) or use bfs_run, which
 * returns BFS_ERR_TIMEOUT.
 */
bfs_status bfs_run_csr_noalloc(const int64_t* row_offsets, const int32_t* col_ids, int64_t n, int64_t nnz,
                               int32_t root, int32_t* parent_dev, int32_t* level_dev, void* stream);

/*
 * Autotuner: times bfs_run (both outputs written) on `k` sample roots
 * (roots_host) for a grid of direction thresholds alpha in {6,14,24,32,96},
 * beta in {12,24,64,128} and top-down hub cut-offs td_big_degree in
 * {64,96,256}; then, from the winner, the top-down chunk size td_chunk in
 * {128,256,512,1024}, then ctas_per_sm in {1, the maximum}, then (CSR,
 * undirected) cluster_size in {1, 8, 16}, one knob at a
 * time.  Each configuration runs once for warm-up, then the k roots timed with
 * CUDA events; the fastest mean goes to *best (other fields from `base`, or
 * the defaults when base is NULL).  Levels do not depend on these choices
 * ("Parallel Direction-Optimizing BFS": the heuristic only picks the cheaper
 * direction; the launch knobs only split the work).  Synchronises `stream`;
 * *best_ms receives the winner's mean time per search (may be NULL).  Errors:
 * INVALID, CUDA, TIMEOUT.
 */
bfs_status bfs_autotune(bfs_graph* g, const int32_t* roots_host, int32_t k, const bfs_options* base,
                        bfs_options* best, double* best_ms, void* stream);

/* Wait for the graph's enqueued searches; returns the first device-side error since the last sync. */
bfs_status bfs_graph_sync(bfs_graph* g, void* stream);

/*
 * Testing only (failure detection without a fault): every grid barrier of the
 * graph's later searches waits for `extra` arrivals that never come, so each
 * wait runs out after the search's timeout_ms and the search returns
 * BFS_ERR_TIMEOUT with the device context intact.  0 turns it off.  INVALID
 * for extra < 0 or a NULL graph.
 */
bfs_status bfs_debug_set_barrier_extra(bfs_graph* g, int32_t extra);

/* ----------------------------------------------------------------- server */

/*
 * A query server that keeps graphs resident and runs BFS queries with
 * continuous batching: each graph has up to max_lanes (<= 64) lane slots of a
 * running multi-source search; a query is admitted into a free slot at the
 * next level boundary (its lane starts at the current iteration, and its
 * levels count from there), so queries that arrive while others run share
 * the device work.  Each graph also keeps up to four plain single-source
 * search states that take queued queries first (plain searches); lanes open
 * for the overflow once 8 or more queries wait, and keep admitting while they
 * run.  A graph whose probe search at
 * add time needs more than 128 levels (large diameter, e.g. a torus) is served
 * by up to 8 plain searches running side by side, each on one 16-CTA
 * thread-block cluster (cluster levels), instead of lanes.  Levels are the same on every path.  Admission is bounded by
 * hbm_budget_bytes for per-query state and search states.  A host thread
 * drives the device; outputs land in caller memory.
 */
bfs_status bfs_server_create(int64_t hbm_budget_bytes, int32_t max_lanes, bfs_server** out);

/*
 * The same with an allocator: every device buffer the server owns (per-slot
 * lane masks, queues and control blocks, the plain-search executors' work
 * buffers) comes from `alloc` (NULL: cudaMalloc / cudaFree).  The hook must stay
 * valid until bfs_server_destroy returns.
 */
bfs_status bfs_server_create_ex(int64_t hbm_budget_bytes, int32_t max_lanes, const bfs_allocator* alloc,
                                bfs_server** out);

/* Make `g` servable (the server does not own it; keep it alive until destroy). */
bfs_status bfs_server_add_graph(bfs_server* s, bfs_graph* g, int32_t* slot);

/*
 * Queue a query (graph slot, root).  level_out_host: caller-owned host array
 * of the graph's n int32, filled with the levels when the ticket completes
 * (must stay valid until then).  Never blocks; BUSY if the request queue is
 * full, INVALID for a bad slot/root.
 */
bfs_status bfs_submit(bfs_server* s, int32_t slot, int32_t root, int32_t* level_out_host, uint64_t* ticket);

/* BFS_OK when done (result written), BFS_ERR_NOT_READY while in flight, INVALID for an unknown ticket. */
bfs_status bfs_poll(bfs_server* s, uint64_t ticket);

/* Block until done or timeout_ms elapsed (NOT_READY); timeout_ms < 0 waits forever. */
bfs_status bfs_wait(bfs_server* s, uint64_t ticket, int64_t timeout_ms);

/*
 * Latency of completed tickets in microseconds (submit -> done), and counters:
 * out[0] completed, out[1] device launches, out[2] lanes filled summed over launches.
 */
bfs_status bfs_server_stats(bfs_server* s, int64_t* counters3);
bfs_status bfs_ticket_latency_us(bfs_server* s, uint64_t ticket, double* us);

void bfs_server_destroy(bfs_server* s);

/* ----------------------------------------------------------------- misc */

const char* bfs_status_string(bfs_status st);
const char* bfs_last_error(void);
/* Library version string. */
const char* bfs_version(void);

#ifdef __cplusplus
}
#endif
#endif
