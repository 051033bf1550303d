// server.cpp -- BFS query server with continuous batching.
//
// Graphs stay resident.  Each graph slot runs one multi-source search state
// (64 lane bits per vertex, see bfs_multi.cu) that advances level by level;
// a query is a (slot, root) pair.  A host worker thread loops:
//   1. admission: queued queries of a slot take free lanes, bounded by
//      max_lanes and by the HBM budget (each lane needs a device row of n
//      int32 for its levels; rows are allocated on first use and kept);
//      a new lane starts at the slot's current iteration, so it joins the
//      running batch at a level boundary;
//   2. one level of every slot that has active lanes, each slot on its own
//      stream so the levels of different graphs overlap on the device;
//   3. completion: a lane whose frontier came back empty is finished; its row
//      is copied to the caller's host buffer and the ticket completes.
// Level values of a lane count from its own start, so a query gets the same
// levels whether it ran alone or in a mix (tested).
//
// Lanes pay off only when many queries of a graph are in flight: a 64-lane
// search with one or two lanes busy costs several plain searches.  Every slot
// therefore also owns a few executors, each a single-source search state with
// its own stream; free executors take queued queries first (plain searches),
// and lanes take the overflow: a slot opens lanes once kLaneBatch queries wait
// (and keeps admitting into them while they run).  Graphs of large diameter (a
// probe search at add time takes more than kDeepLevels levels, e.g. a torus)
// gain nothing from lanes -- their levels are short and many, and every lane
// pays every level -- so their slots use kDeepExecs executors with small grids
// only; those cooperative launches run side by side, each bound by its own
// level latency rather than by the device's throughput.  A deep executor's grid
// is one thread-block cluster (kDeepGrid CTAs): its small levels run as cluster
// levels whatever the grid, and the CTAs it does not hold stay free for the
// other slots' launches.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bfs_internal.h"
#include "bfs_multi.h"

using namespace bfsrt;
using Clock = std::chrono::steady_clock;

namespace {

enum TicketState { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3 };

constexpr int kMinCtas = 8;   // smallest grid of a slot's launch
constexpr int kDeepLevels = 128;   // probe levels above which a slot runs concurrent single searches
constexpr int kDeepExecs = 8;      // concurrent single-source searches of such a slot
constexpr int kDeepGrid = 16;      // CTAs of each (one cluster of 16)
constexpr int kExecs = 4;          // executors of every other slot
constexpr size_t kLaneBatch = 8;   // a queue this long (or busy lanes) sends queries to lanes

struct Ticket {
    int slot = 0;
    int root = 0;
    int32_t* host_out = nullptr;
    int state = kQueued;
    bfs_status err = BFS_OK;
    int lane = -1;
    Clock::time_point t_submit, t_done;
};

struct Lane {
    bool busy = false;        // holds a query (running, or its row is being copied out)
    uint64_t ticket = 0;
    int32_t* row = nullptr;   // device [n]
};

struct CopyBatch {
    cudaEvent_t ev = nullptr;
    std::vector<uint64_t> tickets;
};

// One single-source search in flight of a deep slot.
struct Exec {
    SingleWork w;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    int32_t* dlevel = nullptr;    // device [n]
    void* ctrl_pinned = nullptr;  // host copy of the search's control block (status)
    uint64_t ticket = 0;
    bool busy = false;
};

struct Slot {
    bfs_graph* g = nullptr;
    bool deep = false;                   // queries run as concurrent single-source searches (execs)
    std::vector<Exec*> execs;
    MultiWork w;
    cudaStream_t stream = nullptr;       // levels of this slot
    cudaStream_t copy_stream = nullptr;  // result rows to host
    cudaEvent_t ev = nullptr;            // end of the launch in flight
    std::vector<unsigned char> table;    // host mirror of the lane table
    Lane lanes[64];
    unsigned long long active = 0;       // lanes with a search in progress
    unsigned long long stale = 0;        // finished lanes whose bits are still in seen/front
    unsigned long long admitted = 0;     // lanes admitted for the next launch
    int iter = 0;
    bool running = false;
    int max_iters = 64;
    bfsk::MCtrl* ctrl_pinned = nullptr;
    std::deque<uint64_t> queue;
    std::deque<CopyBatch> copies;
    std::vector<cudaEvent_t> spare_events;
};

}  // namespace

struct bfs_server {
    bfsrt::DeviceAlloc mem;   // every device buffer the server owns (hook or cudaMalloc)
    int64_t budget = 0;
    int64_t used = 0;
    int32_t max_lanes = 64;
    int device = 0;
    int total_ctas = 0;
    std::vector<Slot*> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::unordered_map<uint64_t, Ticket> tickets;
    uint64_t next_ticket = 1;
    size_t queue_cap = 1 << 22;
    size_t queued = 0;
    bool stop = false;
    std::thread worker;
    int64_t completed = 0, launches = 0, lanes_filled = 0;
    std::string fatal;
};

namespace {

void fail_slot(bfs_server* sv, Slot& s, const std::string& why) {
    for (int i = 0; i < 64; i++) {
        if (!s.lanes[i].busy) continue;
        auto it = sv->tickets.find(s.lanes[i].ticket);
        if (it != sv->tickets.end()) {
            it->second.state = kFailed;
            it->second.err = BFS_ERR_CUDA;
            it->second.t_done = Clock::now();
        }
        s.lanes[i].busy = false;
    }
    s.active = 0;
    s.admitted = 0;
    s.running = false;
    sv->fatal = why;
}

cudaEvent_t take_event(Slot& s) {
    if (!s.spare_events.empty()) {
        cudaEvent_t e = s.spare_events.back();
        s.spare_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
}

// Executors of a slot: complete finished searches and, if `start`, put queued
// queries on the free ones.
bool step_execs(bfs_server* sv, Slot& s, bool start) {
    bool progress = false;
    for (Exec* ex : s.execs) {
        if (ex->busy) {
            const cudaError_t q = cudaEventQuery(ex->ev);
            if (q == cudaErrorNotReady) continue;
            const bool ok = q == cudaSuccess && single_ctrl_status(ex->ctrl_pinned) == 0;
            if (q != cudaSuccess) (void)cudaGetLastError();
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                Ticket& t = sv->tickets[ex->ticket];
                t.state = ok ? kDone : kFailed;
                t.err = ok ? BFS_OK : (q != cudaSuccess ? BFS_ERR_CUDA : BFS_ERR_TIMEOUT);
                t.t_done = Clock::now();
                if (!ok) sv->fatal = q != cudaSuccess ? cudaGetErrorString(q) : "device status error (barrier timeout)";
                sv->completed++;
            }
            ex->busy = false;
            progress = true;
            sv->cv_done.notify_all();
        }
        if (!start || ex->busy) continue;
        uint64_t tk = 0;
        int root = 0;
        int32_t* out = nullptr;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            if (s.queue.empty()) continue;   // still look at the other searches in flight
            tk = s.queue.front();
            s.queue.pop_front();
            sv->queued--;
            Ticket& t = sv->tickets[tk];
            t.state = kRunning;
            root = t.root;
            out = t.host_out;
        }
        bfs_options o;
        bfs_options_default(&o);
        if (s.g->cols_hf) o.bu_rows = BFS_BU_ROWS_HUB_FIRST;
        bfs_status st = single_launch_work(s.g, ex->w, &root, 1, nullptr, ex->dlevel, o, ex->stream);
        if (st == BFS_OK &&
            (cudaMemcpyAsync(ex->ctrl_pinned, ex->w.ctrl, single_ctrl_bytes(), cudaMemcpyDeviceToHost, ex->stream) !=
                 cudaSuccess ||
             cudaMemcpyAsync(out, ex->dlevel, sizeof(int32_t) * (size_t)s.g->n, cudaMemcpyDeviceToHost, ex->stream) !=
                 cudaSuccess ||
             cudaEventRecord(ex->ev, ex->stream) != cudaSuccess))
            st = BFS_ERR_CUDA;
        if (st != BFS_OK) {
            std::lock_guard<std::mutex> lk(sv->mu);
            Ticket& t = sv->tickets[tk];
            t.state = kFailed;
            t.err = st;
            t.t_done = Clock::now();
            sv->fatal = bfs_last_error();
            sv->cv_done.notify_all();
            continue;
        }
        ex->ticket = tk;
        ex->busy = true;
        progress = true;
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->launches++;
        sv->lanes_filled++;
    }
    return progress;
}

// Worker loop.  Slots progress independently: a slot whose launch ended is
// harvested (finished lanes -> rows copied out on the copy stream), refilled
// from its queue (new lanes join at this level boundary) and relaunched; a
// slot still running is skipped.  No slot waits for another.
void worker_main(bfs_server* sv) {
    cudaSetDevice(sv->device);
    std::vector<Slot*> snap;
    while (true) {
        bool progress = false;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            auto has_work = [&] {
                for (Slot* s : sv->slots) {
                    if (s->running || s->active || !s->queue.empty() || !s->copies.empty()) return true;
                    for (Exec* ex : s->execs)
                        if (ex->busy) return true;
                }
                return false;
            };
            sv->cv_work.wait(lk, [&] { return sv->stop || has_work(); });
            if (sv->stop) break;
            snap = sv->slots;   // slots are only appended
        }
        // slots with work share the device's co-resident CTAs equally, so that
        // their cooperative launches always fit side by side
        int busy = 0;
        for (Slot* sp : snap) busy += (sp->running || sp->active || !sp->queue.empty()) ? 1 : 0;
        for (Slot* sp : snap) {
            Slot& s = *sp;
            if (s.deep) {
                progress |= step_execs(sv, s, true);
                continue;
            }
            // free executors take queued queries first (plain searches); lanes take the
            // overflow: new lanes open only when kLaneBatch queries wait or lanes are running
            progress |= step_execs(sv, s, true);
            // ---------------------------------------------- harvest a finished launch
            if (s.running) {
                const cudaError_t q = cudaEventQuery(s.ev);
                if (q == cudaErrorNotReady) continue;
                s.running = false;
                progress = true;
                const bfsk::MCtrl& c = *s.ctrl_pinned;
                if (q != cudaSuccess || c.b.status != 0) {
                    (void)cudaGetLastError();
                    std::lock_guard<std::mutex> lk(sv->mu);
                    fail_slot(sv, s, q != cudaSuccess ? cudaGetErrorString(q) : "device status error (barrier timeout)");
                    cudaMemsetAsync(s.w.ctrl, 0, sizeof(bfsk::MCtrl), s.stream);
                    continue;
                }
                s.iter += (int)c.s_done;
                const unsigned long long finished = s.active & c.s_finished;
                const unsigned long long all_done = (c.s_nf == 0) ? s.active : 0ull;
                const unsigned long long ended = finished | all_done;
                if (ended) {
                    CopyBatch cb;
                    cb.ev = take_event(s);
                    cudaEventRecord(s.ev, s.stream);
                    cudaStreamWaitEvent(s.copy_stream, s.ev, 0);
                    std::lock_guard<std::mutex> lk(sv->mu);
                    for (int i = 0; i < 64; i++) {
                        if (!((ended >> i) & 1ull)) continue;
                        Lane& L = s.lanes[i];
                        cudaMemcpyAsync(sv->tickets[L.ticket].host_out, L.row, sizeof(int32_t) * (size_t)s.g->n,
                                        cudaMemcpyDeviceToHost, s.copy_stream);
                        cb.tickets.push_back(L.ticket);
                    }
                    if (cb.ev) cudaEventRecord(cb.ev, s.copy_stream);
                    s.copies.push_back(cb);
                    s.active &= ~ended;
                    s.stale |= ended;
                }
            }
            // ---------------------------------------------- complete copied results
            while (!s.copies.empty()) {
                CopyBatch& cb = s.copies.front();
                const cudaError_t q = cb.ev ? cudaEventQuery(cb.ev) : cudaStreamSynchronize(s.copy_stream);
                if (q == cudaErrorNotReady) break;
                progress = true;
                {
                    std::lock_guard<std::mutex> lk(sv->mu);
                    const auto now = Clock::now();
                    for (uint64_t tk : cb.tickets) {
                        Ticket& t = sv->tickets[tk];
                        t.state = q == cudaSuccess ? kDone : kFailed;
                        t.err = q == cudaSuccess ? BFS_OK : BFS_ERR_CUDA;
                        t.t_done = now;
                        s.lanes[t.lane].busy = false;
                        sv->completed++;
                    }
                }
                if (cb.ev) s.spare_events.push_back(cb.ev);
                s.copies.pop_front();
                sv->cv_done.notify_all();
            }
            if (s.running) continue;
            // ---------------------------------------------- admission at this level boundary
            unsigned long long newmask = 0;
            {
                std::lock_guard<std::mutex> lk(sv->mu);
                const size_t row_bytes = sizeof(int32_t) * (size_t)s.g->n;
                const bool open_lanes = s.active || s.queue.size() >= kLaneBatch || s.execs.empty();
                for (int i = 0; open_lanes && i < sv->max_lanes && !s.queue.empty(); i++) {
                    Lane& L = s.lanes[i];
                    if (L.busy) continue;
                    if (!L.row) {
                        if (sv->used + (int64_t)row_bytes > sv->budget) break;   // admission bounded by HBM budget
                        L.row = (int32_t*)sv->mem.alloc(row_bytes, s.stream);
                        if (!L.row) {
                            (void)cudaGetLastError();
                            break;
                        }
                        sv->used += (int64_t)row_bytes;
                    }
                    const uint64_t tk = s.queue.front();
                    s.queue.pop_front();
                    sv->queued--;
                    Ticket& t = sv->tickets[tk];
                    t.state = kRunning;
                    t.lane = i;
                    L.busy = true;
                    L.ticket = tk;
                    ms_lane_table_set(s.table.data(), i, L.row, s.iter, t.root);
                    newmask |= 1ull << i;
                }
            }
            if (!s.active && !newmask) continue;
            // ---------------------------------------------- launch the next levels
            const unsigned long long drop = s.stale & newmask;
            s.stale &= ~newmask;
            s.active |= newmask;
            const int share = std::max(kMinCtas, sv->total_ctas / std::max(1, busy));
            const int by_size = (int)std::max<long long>(kMinCtas, s.g->n >> 15);
            const int grid = std::min(share, by_size);
            bfs_status st = ms_serve_launch(s.g, s.w, s.table.data(), newmask, drop, s.active, s.iter, s.max_iters,
                                            grid, s.ctrl_pinned, s.stream);
            if (st == BFS_OK && cudaEventRecord(s.ev, s.stream) != cudaSuccess) st = BFS_ERR_CUDA;
            if (st != BFS_OK) {
                std::lock_guard<std::mutex> lk(sv->mu);
                fail_slot(sv, s, bfs_last_error());
                continue;
            }
            s.running = true;
            progress = true;
            sv->launches++;
            sv->lanes_filled += __builtin_popcountll(s.active);
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
}

// Levels of one search from the first vertex with neighbours (0 if the graph has none).
bfs_status probe_levels(bfs_graph* g, bfsrt::DeviceAlloc* mem, int* levels) {
    *levels = 0;
    const long long words = std::min<long long>(g->W, 1 << 16);
    std::vector<uint32_t> iso((size_t)words);
    if (cudaMemcpy(iso.data(), g->isolated, sizeof(uint32_t) * (size_t)words, cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_fail(cudaGetLastError(), "probe: isolated bitmap");
    int root = -1;
    for (long long w = 0; w < words && root < 0; w++)
        if (iso[(size_t)w] != 0xFFFFFFFFu) root = (int)(w * 32 + __builtin_ctz(~iso[(size_t)w]));
    if (root < 0) return BFS_OK;
    const size_t lv_bytes = sizeof(int32_t) * (size_t)g->n;
    int32_t* lv = (int32_t*)mem->alloc(lv_bytes, nullptr);
    if (!lv) return fail(BFS_ERR_OOM, "probe: level buffer");
    bfs_level_record recs[1];
    bfs_stats st;
    memset(&st, 0, sizeof st);
    st.levels = recs;
    st.levels_capacity = 1;
    const bfs_status r = bfs_run(g, root, nullptr, lv, nullptr, nullptr, &st);
    if (cudaDeviceSynchronize() != cudaSuccess) (void)cudaGetLastError();
    mem->release(lv, lv_bytes, nullptr);
    if (r != BFS_OK) return r;
    *levels = st.num_levels;
    return BFS_OK;
}

// Up to `count` executors with launch grid `grid`, as many as the HBM budget
// leaves room for; fewer than `min_count` is an error.
bfs_status add_execs(bfs_server* sv, Slot* s, int count, int grid, int min_count) {
    const int64_t row = (int64_t)sizeof(int32_t) * s->g->n;
    // a search state holds two vertex queues, the level staging, the hub tasks and bitmaps
    const int64_t state = 9 * s->g->n + 20 * s->g->nnz / 64 + (1 << 22);
    for (int i = 0; i < count; i++) {
        if (sv->used + row + state > sv->budget) {
            if (i >= min_count) return BFS_OK;
            return fail(BFS_ERR_OOM, "HBM budget too small for the search executors");
        }
        Exec* ex = new (std::nothrow) Exec();
        if (!ex) return fail(BFS_ERR_OOM, "host allocation of a search executor");
        s->execs.push_back(ex);
        if (cudaStreamCreateWithFlags(&ex->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&ex->ev, cudaEventDisableTiming) != cudaSuccess)
            return fail(BFS_ERR_CUDA, "search executor stream / event");
        if (cudaMallocHost(&ex->ctrl_pinned, single_ctrl_bytes()) != cudaSuccess)
            return fail(BFS_ERR_OOM, "search executor control copy");
        ex->dlevel = (int32_t*)sv->mem.alloc((size_t)row, ex->stream);
        if (!ex->dlevel) return fail(BFS_ERR_OOM, "search executor level buffer");
        ex->w.mem = &sv->mem;
        bfs_status r = single_prepare_work(s->g, ex->w, ex->stream, grid);
        if (r != BFS_OK) return r;
        if (cudaStreamSynchronize(ex->stream) != cudaSuccess) return fail(BFS_ERR_CUDA, "search executor setup");
        sv->used += row + (int64_t)ex->w.bytes;
    }
    return BFS_OK;
}

void free_execs(bfs_server* sv, Slot* s) {
    for (Exec* ex : s->execs) {
        if (ex->stream) cudaStreamSynchronize(ex->stream);
        single_release_work(s->g, ex->w);
        if (ex->dlevel) sv->mem.release(ex->dlevel, sizeof(int32_t) * (size_t)s->g->n, ex->stream);
        if (ex->ctrl_pinned) cudaFreeHost(ex->ctrl_pinned);
        if (ex->ev) cudaEventDestroy(ex->ev);
        if (ex->stream) cudaStreamDestroy(ex->stream);
        delete ex;
    }
    s->execs.clear();
}

}  // namespace

extern "C" {

bfs_status bfs_server_create(int64_t hbm_budget_bytes, int32_t max_lanes, bfs_server** out) {
    return bfs_server_create_ex(hbm_budget_bytes, max_lanes, nullptr, out);
}

bfs_status bfs_server_create_ex(int64_t hbm_budget_bytes, int32_t max_lanes, const bfs_allocator* alloc,
                                bfs_server** out) {
    if (!out) return fail(BFS_ERR_INVALID, "out handle pointer is NULL");
    *out = nullptr;
    if (alloc && (!alloc->alloc || !alloc->free))
        return fail(BFS_ERR_INVALID, "allocator hook needs both alloc and free");
    if (hbm_budget_bytes <= 0) return fail(BFS_ERR_INVALID, "hbm_budget_bytes must be > 0");
    if (max_lanes < 1 || max_lanes > 64) return fail(BFS_ERR_INVALID, "max_lanes must lie in [1, 64]");
    bfs_server* sv = new (std::nothrow) bfs_server();
    if (!sv) return fail(BFS_ERR_OOM, "host allocation of the server");
    sv->budget = hbm_budget_bytes;
    sv->max_lanes = max_lanes;
    if (alloc) {
        sv->mem.hook = *alloc;
        sv->mem.has_hook = true;
    }
    cudaError_t e = cudaGetDevice(&sv->device);
    if (e != cudaSuccess) {
        delete sv;
        return cuda_fail(e, "cudaGetDevice");
    }
    sv->worker = std::thread(worker_main, sv);
    *out = sv;
    return BFS_OK;
}

bfs_status bfs_server_add_graph(bfs_server* sv, bfs_graph* g, int32_t* slot) {
    if (!sv || !g) return fail(BFS_ERR_INVALID, "NULL server or graph");
    if (g->directed) return fail(BFS_ERR_UNSUPPORTED, "server: undirected graphs only");
    std::lock_guard<std::mutex> lk(sv->mu);
    Slot* s = new (std::nothrow) Slot();
    if (!s) return fail(BFS_ERR_OOM, "host allocation of a slot");
    s->g = g;
    int deep_levels = 0;
    bfs_status pr = probe_levels(g, &sv->mem, &deep_levels);
    if (pr != BFS_OK) {
        delete s;
        return fail(pr, std::string("server: add_graph: probe search: ") + bfs_last_error());
    }
    if (deep_levels > kDeepLevels) {
        s->deep = true;
        bfs_status r = add_execs(sv, s, kDeepExecs, kDeepGrid, 1);
        if (r != BFS_OK) {
            std::string msg = bfs_last_error();
            free_execs(sv, s);
            delete s;
            return fail(r, "server: add_graph: " + msg);
        }
        sv->slots.push_back(s);
        if (slot) *slot = (int32_t)(sv->slots.size() - 1);
        return BFS_OK;
    }
    const int64_t need = (int64_t)(3 * sizeof(unsigned long long) * (size_t)g->n);
    if (sv->used + need > sv->budget) {
        delete s;
        return fail(BFS_ERR_OOM, "HBM budget too small for the graph's lane masks");
    }
    cudaStream_t st = nullptr, cst = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cst, cudaStreamNonBlocking) != cudaSuccess) {
        if (st) cudaStreamDestroy(st);
        delete s;
        return fail(BFS_ERR_CUDA, "cudaStreamCreate");
    }
    s->stream = st;
    s->copy_stream = cst;
    s->w.mem = &sv->mem;
    bfs_status r = multi_alloc(g, s->w, st);
    if (r == BFS_OK) r = ms_serve_reset(g, s->w, st);
    if (r == BFS_OK && cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming) != cudaSuccess) r = BFS_ERR_CUDA;
    if (r == BFS_OK && cudaMallocHost((void**)&s->ctrl_pinned, sizeof(bfsk::MCtrl)) != cudaSuccess) r = BFS_ERR_OOM;
    if (r == BFS_OK && cudaStreamSynchronize(st) != cudaSuccess) r = BFS_ERR_CUDA;
    if (r != BFS_OK) {
        std::string msg = bfs_last_error();
        multi_free(g, s->w);
        if (s->ev) cudaEventDestroy(s->ev);
        if (s->ctrl_pinned) cudaFreeHost(s->ctrl_pinned);
        cudaStreamDestroy(st);
        cudaStreamDestroy(cst);
        delete s;
        return fail(r, "server: add_graph: " + msg);
    }
    if (sv->total_ctas == 0) sv->total_ctas = ms_serve_max_grid(g, s->w);
    {
        // plain searches of this graph: about one CTA per 32K vertices, up to half the device
        const int grid = (int)std::min<long long>(std::max<long long>(kMinCtas, g->n >> 15), sv->total_ctas / 2);
        bfs_status r = add_execs(sv, s, kExecs, grid, 0);
        if (r != BFS_OK) {
            std::string msg = bfs_last_error();
            free_execs(sv, s);
            multi_free(g, s->w);
            cudaEventDestroy(s->ev);
            cudaFreeHost(s->ctrl_pinned);
            cudaStreamDestroy(s->stream);
            cudaStreamDestroy(s->copy_stream);
            delete s;
            return fail(r, "server: add_graph: " + msg);
        }
    }
    memset(s->ctrl_pinned, 0, sizeof(bfsk::MCtrl));
    s->table.assign(ms_lane_table_bytes(), 0);
    sv->used += (int64_t)s->w.bytes;
    sv->slots.push_back(s);
    if (slot) *slot = (int32_t)(sv->slots.size() - 1);
    return BFS_OK;
}

bfs_status bfs_submit(bfs_server* sv, int32_t slot, int32_t root, int32_t* level_out_host, uint64_t* ticket) {
    if (!sv || !ticket || !level_out_host) return fail(BFS_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (slot < 0 || (size_t)slot >= sv->slots.size()) return fail(BFS_ERR_INVALID, "unknown graph slot");
    Slot& s = *sv->slots[slot];
    if (root < 0 || (int64_t)root >= s.g->n) return fail(BFS_ERR_INVALID, "root outside [0, n)");
    if (sv->queued >= sv->queue_cap) return fail(BFS_ERR_BUSY, "request queue is full");
    const uint64_t tk = sv->next_ticket++;
    Ticket t;
    t.slot = slot;
    t.root = root;
    t.host_out = level_out_host;
    t.t_submit = Clock::now();
    sv->tickets[tk] = t;
    s.queue.push_back(tk);
    sv->queued++;
    *ticket = tk;
    sv->cv_work.notify_one();
    return BFS_OK;
}

bfs_status bfs_poll(bfs_server* sv, uint64_t ticket) {
    if (!sv) return fail(BFS_ERR_INVALID, "NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return fail(BFS_ERR_INVALID, "unknown ticket");
    if (it->second.state == kDone) return BFS_OK;
    if (it->second.state == kFailed) return fail(it->second.err, "query failed: " + sv->fatal);
    return BFS_ERR_NOT_READY;
}

bfs_status bfs_wait(bfs_server* sv, uint64_t ticket, int64_t timeout_ms) {
    if (!sv) return fail(BFS_ERR_INVALID, "NULL server");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return fail(BFS_ERR_INVALID, "unknown ticket");
    auto ready = [&] { return it->second.state == kDone || it->second.state == kFailed; };
    if (timeout_ms < 0) {
        sv->cv_done.wait(lk, ready);
    } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        return BFS_ERR_NOT_READY;
    }
    if (it->second.state == kFailed) return fail(it->second.err, "query failed: " + sv->fatal);
    return BFS_OK;
}

bfs_status bfs_server_stats(bfs_server* sv, int64_t* counters3) {
    if (!sv || !counters3) return fail(BFS_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    counters3[0] = sv->completed;
    counters3[1] = sv->launches;
    counters3[2] = sv->lanes_filled;
    return BFS_OK;
}

bfs_status bfs_ticket_latency_us(bfs_server* sv, uint64_t ticket, double* us) {
    if (!sv || !us) return fail(BFS_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return fail(BFS_ERR_INVALID, "unknown ticket");
    if (it->second.state != kDone) return BFS_ERR_NOT_READY;
    *us = std::chrono::duration<double, std::micro>(it->second.t_done - it->second.t_submit).count();
    return BFS_OK;
}

void bfs_server_destroy(bfs_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (Slot* s : sv->slots) {
        if (s->deep) {
            free_execs(sv, s);
            delete s;
            continue;
        }
        free_execs(sv, s);
        cudaStreamSynchronize(s->stream);
        cudaStreamSynchronize(s->copy_stream);
        for (auto& L : s->lanes)
            if (L.row) sv->mem.release(L.row, sizeof(int32_t) * (size_t)s->g->n, s->stream);
        multi_free(s->g, s->w);
        cudaEventDestroy(s->ev);
        for (auto& cb : s->copies)
            if (cb.ev) cudaEventDestroy(cb.ev);
        for (auto e : s->spare_events) cudaEventDestroy(e);
        cudaFreeHost(s->ctrl_pinned);
        cudaStreamDestroy(s->stream);
        cudaStreamDestroy(s->copy_stream);
        delete s;
    }
    for (auto& kv : sv->tickets)
        if (kv.second.state == kQueued || kv.second.state == kRunning) kv.second.state = kFailed;
    sv->cv_done.notify_all();
    delete sv;
}

}  // extern "C"
