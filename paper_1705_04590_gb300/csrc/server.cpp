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

struct Slot {
    bfs_graph* g = nullptr;
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
                for (Slot* s : sv->slots)
                    if (s->running || s->active || !s->queue.empty() || !s->copies.empty()) return true;
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
                for (int i = 0; i < sv->max_lanes && !s.queue.empty(); i++) {
                    Lane& L = s.lanes[i];
                    if (L.busy) continue;
                    if (!L.row) {
                        if (sv->used + (int64_t)row_bytes > sv->budget) break;   // admission bounded by HBM budget
                        if (cudaMalloc(&L.row, row_bytes) != cudaSuccess) {
                            (void)cudaGetLastError();
                            L.row = nullptr;
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

}  // namespace

extern "C" {

bfs_status bfs_server_create(int64_t hbm_budget_bytes, int32_t max_lanes, bfs_server** out) {
    if (!out) return fail(BFS_ERR_INVALID, "out handle pointer is NULL");
    *out = nullptr;
    if (hbm_budget_bytes <= 0) return fail(BFS_ERR_INVALID, "hbm_budget_bytes must be > 0");
    if (max_lanes < 1 || max_lanes > 64) return fail(BFS_ERR_INVALID, "max_lanes must lie in [1, 64]");
    bfs_server* sv = new (std::nothrow) bfs_server();
    if (!sv) return fail(BFS_ERR_OOM, "host allocation of the server");
    sv->budget = hbm_budget_bytes;
    sv->max_lanes = max_lanes;
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
    std::lock_guard<std::mutex> lk(sv->mu);
    Slot* s = new (std::nothrow) Slot();
    if (!s) return fail(BFS_ERR_OOM, "host allocation of a slot");
    s->g = g;
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
        cudaStreamSynchronize(s->stream);
        cudaStreamSynchronize(s->copy_stream);
        for (auto& L : s->lanes)
            if (L.row) cudaFree(L.row);
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
