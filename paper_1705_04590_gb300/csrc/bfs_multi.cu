// bfs_multi.cu -- batched multi-source BFS over 64-bit per-vertex lane masks.
//
// Up to 64 searches advance together.  Lane i of vertex v is bit i of three
// masks: seen[v] (lane i has reached v), front[v] (v is in lane i's current
// frontier), next[v] (v joins lane i's next frontier).  One level of all
// lanes at once, in either direction of "Parallel Direction-Optimizing BFS":
//   top-down  (push, the per-lane Algorithm 1 step): for v with front[v] != 0,
//             for u in adj(v): next[u] |= front[v] & ~seen[u]  (64-bit atomicOr)
//   bottom-up (pull, the per-lane Algorithm 2 step): for u with lanes missing
//             (miss = active & ~seen[u]): OR front[v] over adj(u) in order and
//             stop once every missing lane is covered; next[u] = acc & miss
//   apply:    seen |= next, front = next, next = 0; for each new lane bit i of
//             v: level_i[v] = iteration + 1 - start_i.
// Direction per iteration from the union frontier with the same rule as the
// single-source search (m_f * alpha > m_u; n_f * beta < n).  Levels do not
// depend on it.
//
// Two drivers share these phases:
//  * bfs_multi_kernel: one persistent cooperative launch for a batch of <= 64
//    roots (bfs_run_multi), bounded grid barriers between phases;
//  * ms_*_kernel: one regular launch per phase, stepped by the server so that
//    new lanes can join at a level boundary (continuous batching).
#include <algorithm>
#include <cstring>

#include "bfs_common.cuh"
#include "bfs_internal.h"
#include "bfs_multi.h"

namespace bfsk {

constexpr int kMBlock = 512;
constexpr int kMChunk = 2048;     // edges per top-down chunk task
constexpr unsigned kMFull = 0xffffffffu;

__device__ __forceinline__ long long m_gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long m_gthreads() { return (long long)gridDim.x * blockDim.x; }

__device__ __forceinline__ unsigned long long ldcg64(const unsigned long long* p) { return __ldcg(p); }

__device__ __forceinline__ unsigned long long warp_or64(unsigned long long x) {
    unsigned lo = __reduce_or_sync(kMFull, (unsigned)x);
    unsigned hi = __reduce_or_sync(kMFull, (unsigned)(x >> 32));
    return ((unsigned long long)hi << 32) | lo;
}

// Lane table cached in shared memory by each CTA.
struct LaneSmem {
    int* rows[64];
    int start[64];
};

__device__ __forceinline__ void load_lanes(const MultiParams& p, LaneSmem& L) {
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        L.rows[i] = p.rows[i];
        L.start[i] = p.start[i];
    }
    __syncthreads();
}

// ---------------------------------------------------------------- phases

// Top-down push over vertices with front != 0 (warp-balanced gather; heavy
// rows become chunk tasks processed by ms_tasks_phase after a barrier).
__device__ void ms_td_phase(const MultiParams& p, MCtrl* c, int slot) {
    const int lane = lane_id();
    const long long gw = m_gtid() >> 5, nw = m_gthreads() >> 5;
    for (long long base = gw * 32; base < p.n; base += nw * 32) {
        const long long v = base + lane;
        unsigned long long f = 0;
        long long s = 0, e = 0;
        if (v < p.n) {
            f = ldcg64(p.front + v);
            if (f) {
                s = __ldg(p.off + v);
                e = __ldg(p.off + v + 1);
            }
        }
        const long long deg = e - s;
        int mydeg = 0;
        if (deg > p.big_deg) {
            const long long nch = (deg + kMChunk - 1) / kMChunk;
            const unsigned long long t0 = atomicAdd(&c->ntask[slot], (unsigned long long)nch);
            for (long long k = 0; k < nch; k++) {
                const long long ti = (long long)t0 + k;
                if (ti < p.task_cap) {
                    MTask t;
                    t.start = s + k * kMChunk;
                    t.len = (int)min((long long)kMChunk, e - t.start);
                    t.v = (int)v;
                    p.tasks[ti] = t;
                } else {
                    atomicMax(&c->b.status, kDevOverflow);
                }
            }
        } else {
            mydeg = (int)deg;
        }
        const int incl = warp_inclusive_scan(mydeg);
        const int total = __shfl_sync(kMFull, incl, 31);
        const int excl = incl - mydeg;
        for (int k0 = 0; k0 < total; k0 += 32) {
            const int k = k0 + lane;
            int j = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int cc = __shfl_sync(kMFull, incl, j + step - 1);
                if (cc <= k) j += step;
            }
            const long long sj = __shfl_sync(kMFull, s, j);
            const int exj = __shfl_sync(kMFull, excl, j);
            const unsigned long long fj = __shfl_sync(kMFull, f, j);
            if (k < total) {
                const int u = __ldg(p.cols + sj + (k - exj));
                const unsigned long long nb = fj & ~ldcg64(p.seen + u);
                if (nb) atomicOr(p.next + u, nb);
            }
        }
    }
}

__device__ void ms_tasks_phase(const MultiParams& p, MCtrl* c, int slot) {
    const int lane = lane_id();
    const long long gw = m_gtid() >> 5, nw = m_gthreads() >> 5;
    const long long nt = min((long long)ld_acquire64(&c->ntask[slot]), p.task_cap);
    for (long long t = gw; t < nt; t += nw) {
        const int4 raw = __ldcg(reinterpret_cast<const int4*>(p.tasks + t));
        const long long start = (long long)(unsigned)raw.x | ((long long)raw.y << 32);
        const int len = raw.z, v = raw.w;
        const unsigned long long f = ldcg64(p.front + v);
        for (int k = lane; k < len; k += 32) {
            const int u = __ldg(p.cols + start + k);
            const unsigned long long nb = f & ~ldcg64(p.seen + u);
            if (nb) atomicOr(p.next + u, nb);
        }
    }
}

// Bottom-up pull: a warp owns 32 consecutive vertices; each lane ORs the
// frontier masks of its first 8 neighbours, then rows with lanes still
// missing continue warp-cooperatively 32 neighbours at a time.
__device__ void ms_bu_phase(const MultiParams& p, unsigned long long active) {
    const int lane = lane_id();
    const long long gw = m_gtid() >> 5, nw = m_gthreads() >> 5;
    for (long long base = gw * 32; base < p.n; base += nw * 32) {
        const long long u = base + lane;
        unsigned long long miss = 0, acc = 0;
        long long s = 0, e = 0, pos = 0;
        if (u < p.n) {
            miss = active & ~ldcg64(p.seen + u);
            if (miss) {
                s = __ldg(p.off + u);
                e = __ldg(p.off + u + 1);
                pos = s;   // a degree-0 row has nothing left to scan
            }
        }
        if (miss && e > s) {
            const long long a = s & ~3LL;
            const int4 x0 = __ldg(reinterpret_cast<const int4*>(p.cols + a));
            const int4 x1 = __ldg(reinterpret_cast<const int4*>(p.cols + a + 4));
            const int ids[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
            for (int t = 0; t < 8; t++) {
                const long long q = a + t;
                if (q >= s && q < e) acc |= ldcg64(p.front + ids[t]);
            }
            pos = a + 8;
        }
        unsigned pend = __ballot_sync(kMFull, miss && (acc & miss) != miss && pos < e);
        while (pend) {
            const int L = __ffs(pend) - 1;
            pend &= pend - 1;
            const long long ps = __shfl_sync(kMFull, pos, L), pe = __shfl_sync(kMFull, e, L);
            const unsigned long long mL = __shfl_sync(kMFull, miss, L);
            unsigned long long aL = __shfl_sync(kMFull, acc, L);
            for (long long q0 = ps; q0 < pe; q0 += 32) {
                const long long q = q0 + lane;
                unsigned long long x = 0;
                if (q < pe) x = ldcg64(p.front + __ldg(p.cols + q));
                aL |= warp_or64(x);
                if ((aL & mL) == mL) break;
            }
            if (lane == L) acc = aL;
        }
        const unsigned long long nb = acc & miss;
        if (nb) p.next[u] = nb;
    }
}

// seen |= next, front = next, next = 0, per-lane levels; counts the new
// frontier (n_f, m_f), the degree of vertices every active lane has now seen
// (subtracted from m_u) and which lanes found anything.
__device__ void ms_apply_phase(const MultiParams& p, MCtrl* c, int slot, int iter, unsigned long long active,
                               const LaneSmem& L) {
    const long long tid = m_gtid(), nth = m_gthreads();
    unsigned long long an = 0, am = 0, adone = 0, found = 0;
    for (long long v = tid; v < p.n; v += nth) {
        const unsigned long long x = ldcg64(p.next + v);
        if (x) {
            p.next[v] = 0ull;
            const unsigned long long s = ldcg64(p.seen + v);
            p.seen[v] = s | x;
            p.front[v] = x;
            found |= x;
            const long long deg = __ldg(p.off + v + 1) - __ldg(p.off + v);
            an += 1;
            am += (unsigned long long)deg;
            if ((s & active) != active && ((s | x) & active) == active) adone += (unsigned long long)deg;
            unsigned long long bits = x;
            while (bits) {
                const int i = __ffsll((long long)bits) - 1;
                bits &= bits - 1;
                L.rows[i][v] = iter + 1 - L.start[i];
            }
        } else if (ldcg64(p.front + v)) {
            p.front[v] = 0ull;
        }
    }
    found = warp_or64(found);
    if (lane_id() == 0 && found) atomicOr(&c->found[slot], found);
    block_add4(an, am, adone, 0, &c->accn[slot], &c->accm[slot], &c->mdone[slot], nullptr);
}

// Clear the three masks (grid-stride).
__device__ void ms_clear_phase(const MultiParams& p) {
    const long long tid = m_gtid(), nth = m_gthreads();
    for (long long v = tid; v < p.n; v += nth) {
        p.seen[v] = 0ull;
        p.front[v] = 0ull;
        p.next[v] = 0ull;
    }
}

// Fill the level rows of lanes in `mask` with -1 (rows of n entries).
__device__ void ms_fill_rows(const MultiParams& p, unsigned long long mask, const LaneSmem& L) {
    const long long tid = m_gtid(), nth = m_gthreads();
    unsigned long long bits = mask;
    while (bits) {
        const int i = __ffsll((long long)bits) - 1;
        bits &= bits - 1;
        int* row = L.rows[i];
        for (long long v = tid; v < p.n; v += nth) row[v] = -1;
    }
}

// Seed lanes in `mask` at their roots (atomics: several lanes may share a root).
__device__ void ms_seed_phase(const MultiParams& p, unsigned long long mask, const LaneSmem& L) {
    const long long tid = m_gtid();
    if (tid < 64 && ((mask >> tid) & 1ull)) {
        const int r = p.roots[tid];
        atomicOr(p.seen + r, 1ull << tid);
        atomicOr(p.front + r, 1ull << tid);
        L.rows[tid][r] = 0;
    }
}

__device__ __forceinline__ int ms_decide(const MultiParams& p, int prev, long long nf, long long mf, long long mu) {
    if (p.mode == BFS_MODE_TD_ONLY) return 0;
    if (p.mode == BFS_MODE_BU_ONLY) return 1;
    if (prev == 0) return (mf * (long long)p.alpha > mu) ? 1 : 0;
    return (nf * (long long)p.beta < p.n) ? 0 : 1;
}

// ---------------------------------------------------------------- persistent driver

__global__ void __launch_bounds__(kMBlock, 2) bfs_multi_kernel(MultiParams p) {
    __shared__ LaneSmem L;
    load_lanes(p, L);
    MCtrl* c = p.ctrl;
    const unsigned long long active = p.active;
    ms_clear_phase(p);
    ms_fill_rows(p, active, L);
    if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
    ms_seed_phase(p, active, L);
    if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
    // level-0 frontier statistics from the (few) distinct roots, identical in every CTA
    long long nf = 0, mf = 0, mu = p.nnz;
    for (int i = 0; i < 64; i++) {
        if (!((active >> i) & 1ull)) continue;
        const int r = p.roots[i];
        bool dup = false;
        for (int j = 0; j < i; j++)
            if (((active >> j) & 1ull) && p.roots[j] == r) dup = true;
        if (dup) continue;
        const long long deg = __ldg(p.off + r + 1) - __ldg(p.off + r);
        nf += 1;
        mf += deg;
        if ((ldcg64(p.seen + r) & active) == active) mu -= deg;
    }
    int prev = 0;
    for (int it = 0;; it++) {
        // counters of iteration `it` accumulate in slot it % 3 and are read by
        // every CTA after the closing barrier; the slot of iteration it + 1 is
        // cleared now (its last readers passed a barrier of iteration it - 1)
        const int slot = it % 3, sfree = (it + 1) % 3;
        if (blockIdx.x == 0 && threadIdx.x == 0) c->zero_slot(sfree);
        const int dir = ms_decide(p, prev, nf, mf, mu);
        if (dir == 0) {
            ms_td_phase(p, c, slot);
            if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            if (ld_acquire64(&c->ntask[slot]) > 0) {
                ms_tasks_phase(p, c, slot);
                if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            }
        } else {
            ms_bu_phase(p, active);
            if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
        }
        ms_apply_phase(p, c, slot, it, active, L);
        if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
        const long long nf2 = (long long)ld_acquire64(&c->accn[slot]);
        if (nf2 == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) c->iterations = it + 1;
            break;
        }
        mu -= (long long)ld_acquire64(&c->mdone[slot]);
        nf = nf2;
        mf = (long long)ld_acquire64(&c->accm[slot]);
        prev = dir;
    }
}

// parent_i[v] = min{u in adj(v) : level_i[u] = level_i[v] - 1} (rows sorted: first hit), root -> itself.
__global__ void ms_parent_kernel(MultiParams p, int* const* prow) {
    __shared__ LaneSmem L;
    load_lanes(p, L);
    const long long tid = m_gtid(), nth = m_gthreads();
    for (int i = 0; i < 64; i++) {
        if (!((p.active >> i) & 1ull)) continue;
        const int* lv = L.rows[i];
        int* pr = prow[i];
        for (long long v = tid; v < p.n; v += nth) {
            const int l = lv[v];
            int par = -1;
            if (l == 0) {
                par = (int)v;
            } else if (l > 0) {
                const long long s = __ldg(p.off + v), e = __ldg(p.off + v + 1);
                for (long long k = s; k < e; k++) {
                    const int u = __ldg(p.cols + k);
                    if (lv[u] == l - 1) {
                        par = u;
                        break;
                    }
                }
            }
            pr[v] = par;
        }
    }
}

// ---------------------------------------------------------------- stepped drivers (server)

__global__ void __launch_bounds__(kMBlock) ms_admit_kernel(MultiParams p, unsigned long long newmask) {
    __shared__ LaneSmem L;
    load_lanes(p, L);
    ms_fill_rows(p, newmask, L);
}

__global__ void ms_seed_kernel(MultiParams p, unsigned long long newmask) {
    __shared__ LaneSmem L;
    load_lanes(p, L);
    ms_seed_phase(p, newmask, L);
}

__global__ void __launch_bounds__(kMBlock) ms_clear_kernel(MultiParams p) { ms_clear_phase(p); }

__global__ void __launch_bounds__(kMBlock) ms_td_kernel(MultiParams p, int slot) { ms_td_phase(p, p.ctrl, slot); }

__global__ void __launch_bounds__(kMBlock) ms_tasks_kernel(MultiParams p, int slot) {
    ms_tasks_phase(p, p.ctrl, slot);
}

__global__ void __launch_bounds__(kMBlock) ms_bu_kernel(MultiParams p, unsigned long long active) {
    ms_bu_phase(p, active);
}

__global__ void __launch_bounds__(kMBlock) ms_apply_kernel(MultiParams p, int slot, int iter,
                                                          unsigned long long active) {
    __shared__ LaneSmem L;
    load_lanes(p, L);
    ms_apply_phase(p, p.ctrl, slot, iter, active, L);
}

// Drop lanes in `mask` from every vertex's masks (lanes that finished or are being reused).
__global__ void __launch_bounds__(kMBlock) ms_drop_kernel(MultiParams p, unsigned long long mask) {
    const long long tid = m_gtid(), nth = m_gthreads();
    const unsigned long long keep = ~mask;
    for (long long v = tid; v < p.n; v += nth) {
        const unsigned long long s = p.seen[v];
        if (s & mask) p.seen[v] = s & keep;
        const unsigned long long f = p.front[v];
        if (f & mask) p.front[v] = f & keep;
    }
}

__global__ void ms_zero_slot_kernel(MCtrl* c, int slot) {
    if (threadIdx.x == 0) c->zero_slot(slot);
}

}  // namespace bfsk

// ====================================================================== host

namespace bfsrt {

using bfsk::MCtrl;
using bfsk::MTask;
using bfsk::MultiParams;

static size_t mask_bytes(const bfs_graph* g) { return sizeof(unsigned long long) * (size_t)g->n; }

bfs_status multi_alloc(bfs_graph* g, MultiWork& w, cudaStream_t s) {
    if (w.ready) return BFS_OK;
    const size_t nb = mask_bytes(g);
    const long long task_cap = g->nnz / bfsk::kMChunk + g->nnz / 256 + 1024;
    w.seen = (unsigned long long*)g->mem.alloc(nb, s);
    w.front = (unsigned long long*)g->mem.alloc(nb, s);
    w.next = (unsigned long long*)g->mem.alloc(nb, s);
    w.ctrl = g->mem.alloc(sizeof(MCtrl), s);
    w.tasks = g->mem.alloc(sizeof(MTask) * (size_t)task_cap, s);
    w.lanes = g->mem.alloc(sizeof(bfsk::LaneTable), s);
    w.task_cap = task_cap;
    if (!w.seen || !w.front || !w.next || !w.ctrl || !w.tasks || !w.lanes) {
        w.ready = true;
        multi_free(g, w);
        return fail(BFS_ERR_OOM, "multi-source work buffers: device allocation failed");
    }
    w.bytes = 3 * nb + sizeof(MCtrl) + sizeof(MTask) * (size_t)task_cap + sizeof(bfsk::LaneTable);
    int occ = 0;
    BFS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bfsk::bfs_multi_kernel, bfsk::kMBlock, 0));
    if (occ < 1) return fail(BFS_ERR_UNSUPPORTED, "multi-source kernel cannot be resident");
    w.block = bfsk::kMBlock;
    w.grid = occ * g->sm_count;
    BFS_CUDA_TRY(cudaMemsetAsync(w.ctrl, 0, sizeof(MCtrl), s));
    BFS_CUDA_TRY(cudaMemsetAsync(w.lanes, 0, sizeof(bfsk::LaneTable), s));
    w.ready = true;
    return BFS_OK;
}

void multi_free(bfs_graph* g, MultiWork& w) {
    if (!w.ready) return;
    const size_t nb = mask_bytes(g);
    g->mem.release(w.seen, nb, nullptr);
    g->mem.release(w.front, nb, nullptr);
    g->mem.release(w.next, nb, nullptr);
    g->mem.release(w.ctrl, sizeof(MCtrl), nullptr);
    g->mem.release(w.tasks, sizeof(MTask) * (size_t)w.task_cap, nullptr);
    g->mem.release(w.lanes, sizeof(bfsk::LaneTable), nullptr);
    w = MultiWork();
}

bfs_status multi_prepare(bfs_graph* g, cudaStream_t s) { return multi_alloc(g, g->multi, s); }
void multi_release(bfs_graph* g) { multi_free(g, g->multi); }

static MultiParams multi_params(bfs_graph* g, MultiWork& w, const bfs_options& opt) {
    MultiParams p;
    memset(&p, 0, sizeof p);
    p.off = reinterpret_cast<const long long*>(g->offsets);
    p.cols = g->cols;
    p.n = g->n;
    p.nnz = g->nnz;
    p.seen = w.seen;
    p.front = w.front;
    p.next = w.next;
    p.ctrl = reinterpret_cast<MCtrl*>(w.ctrl);
    p.tasks = reinterpret_cast<MTask*>(w.tasks);
    p.task_cap = w.task_cap;
    bfsk::LaneTable* lt = reinterpret_cast<bfsk::LaneTable*>(w.lanes);
    p.rows = lt->rows;
    p.start = lt->start;
    p.roots = lt->roots;
    p.mode = opt.mode == BFS_MODE_RANDOM ? BFS_MODE_DO : opt.mode;
    p.alpha = opt.alpha;
    p.beta = opt.beta;
    p.big_deg = opt.td_big_degree > 0 ? opt.td_big_degree : 256;
    p.timeout_ns = (unsigned long long)(opt.timeout_ms > 0 ? opt.timeout_ms : 10000) * 1000000ull;
    p.expected = (unsigned)w.grid + (unsigned)(opt.debug_barrier_extra > 0 ? opt.debug_barrier_extra : 0);
    return p;
}

bfs_status multi_launch(bfs_graph* g, const int32_t* roots_host, int32_t k, int32_t* level, int32_t* parent,
                        const bfs_options& opt, cudaStream_t s) {
    MultiWork& w = g->multi;
    for (int32_t c0 = 0; c0 < k; c0 += 64) {
        const int kk = std::min(64, k - c0);
        bfsk::LaneTable t;
        memset(&t, 0, sizeof t);
        for (int i = 0; i < kk; i++) {
            t.rows[i] = level + (size_t)(c0 + i) * (size_t)g->n;
            t.prow[i] = parent ? parent + (size_t)(c0 + i) * (size_t)g->n : nullptr;
            t.start[i] = 0;
            t.roots[i] = roots_host[c0 + i];
        }
        // pageable source: staged by the driver before cudaMemcpyAsync returns,
        // and ordered on the stream before the launch that reads it
        BFS_CUDA_TRY(cudaMemcpyAsync(w.lanes, &t, sizeof t, cudaMemcpyHostToDevice, s));
        BFS_CUDA_TRY(cudaMemsetAsync(w.ctrl, 0, sizeof(MCtrl), s));
        MultiParams p = multi_params(g, w, opt);
        p.active = (kk == 64) ? ~0ull : ((1ull << kk) - 1ull);
        void* args[] = {&p};
        BFS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)bfsk::bfs_multi_kernel, dim3(w.grid), dim3(w.block),
                                                 args, 0, s));
        if (parent) {
            bfsk::LaneTable* lt = reinterpret_cast<bfsk::LaneTable*>(w.lanes);
            bfsk::ms_parent_kernel<<<w.grid, w.block, 0, s>>>(p, lt->prow);
            BFS_CUDA_TRY(cudaGetLastError());
        }
    }
    return BFS_OK;
}

bfs_status multi_collect_status(bfs_graph* g, cudaStream_t s) {
    MCtrl c;
    BFS_CUDA_TRY(cudaMemcpyAsync(&c, g->multi.ctrl, sizeof(MCtrl), cudaMemcpyDeviceToHost, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    if (c.b.status == bfsk::kDevTimeout) return fail(BFS_ERR_TIMEOUT, "multi-source grid barrier ran out of time");
    if (c.b.status == bfsk::kDevOverflow) return fail(BFS_ERR_CUDA, "multi-source task list overflowed");
    return BFS_OK;
}

// ---------------------------------------------------------------- stepped driver (server)

size_t ms_lane_table_bytes() { return sizeof(bfsk::LaneTable); }

void ms_lane_table_set(void* table_host, int lane, int32_t* row, int start, int root) {
    bfsk::LaneTable* t = reinterpret_cast<bfsk::LaneTable*>(table_host);
    t->rows[lane] = row;
    t->prow[lane] = nullptr;
    t->start[lane] = start;
    t->roots[lane] = root;
}

static bfs_options server_opts() {
    bfs_options o;
    bfs_options_default(&o);
    return o;
}

bfs_status ms_step_reset(bfs_graph* g, MultiWork& w, cudaStream_t s) {
    MultiParams p = multi_params(g, w, server_opts());
    bfsk::ms_clear_kernel<<<w.grid, w.block, 0, s>>>(p);
    BFS_CUDA_TRY(cudaGetLastError());
    BFS_CUDA_TRY(cudaMemsetAsync(w.ctrl, 0, sizeof(MCtrl), s));
    return BFS_OK;
}

bfs_status ms_step_admit(bfs_graph* g, MultiWork& w, const void* lane_table_host, unsigned long long newmask,
                         cudaStream_t s) {
    BFS_CUDA_TRY(cudaMemcpyAsync(w.lanes, lane_table_host, sizeof(bfsk::LaneTable), cudaMemcpyHostToDevice, s));
    MultiParams p = multi_params(g, w, server_opts());
    bfsk::ms_admit_kernel<<<w.grid, w.block, 0, s>>>(p, newmask);
    BFS_CUDA_TRY(cudaGetLastError());
    bfsk::ms_seed_kernel<<<1, 64, 0, s>>>(p, newmask);
    BFS_CUDA_TRY(cudaGetLastError());
    return BFS_OK;
}

bfs_status ms_step_drop(bfs_graph* g, MultiWork& w, unsigned long long mask, cudaStream_t s) {
    MultiParams p = multi_params(g, w, server_opts());
    bfsk::ms_drop_kernel<<<w.grid, w.block, 0, s>>>(p, mask);
    BFS_CUDA_TRY(cudaGetLastError());
    return BFS_OK;
}

// One level for every active lane: direction phase(s) then apply; the
// counters of the level are copied into `counters_pinned` (host pinned).
bfs_status ms_step_iterate(bfs_graph* g, MultiWork& w, int iter, int dir, unsigned long long active,
                           void* ctrl_pinned, cudaStream_t s) {
    MultiParams p = multi_params(g, w, server_opts());
    p.active = active;
    const int slot = 0;
    MCtrl* c = reinterpret_cast<MCtrl*>(w.ctrl);
    bfsk::ms_zero_slot_kernel<<<1, 32, 0, s>>>(c, slot);
    BFS_CUDA_TRY(cudaGetLastError());
    if (dir == 0) {
        bfsk::ms_td_kernel<<<w.grid, w.block, 0, s>>>(p, slot);
        BFS_CUDA_TRY(cudaGetLastError());
        bfsk::ms_tasks_kernel<<<w.grid, w.block, 0, s>>>(p, slot);
        BFS_CUDA_TRY(cudaGetLastError());
    } else {
        bfsk::ms_bu_kernel<<<w.grid, w.block, 0, s>>>(p, active);
        BFS_CUDA_TRY(cudaGetLastError());
    }
    bfsk::ms_apply_kernel<<<w.grid, w.block, 0, s>>>(p, slot, iter, active);
    BFS_CUDA_TRY(cudaGetLastError());
    BFS_CUDA_TRY(cudaMemcpyAsync(ctrl_pinned, c, sizeof(MCtrl), cudaMemcpyDeviceToHost, s));
    return BFS_OK;
}

}  // namespace bfsrt
