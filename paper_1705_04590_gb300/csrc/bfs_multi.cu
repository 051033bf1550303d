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
//  * bfs_serve_kernel: one persistent launch per server step that runs levels
//    until a lane finishes (or an iteration cap), so that new lanes can join
//    at a level boundary (continuous batching).
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
//
// The union frontier is kept twice: as masks (front[v] != 0) and as a queue of
// its vertices (fq); the vertices that gain lane bits during a level are
// listed once each in the touched queue (tq), which becomes the next fq.  So a
// top-down level and the apply step cost O(frontier + touched), not O(n); only
// bottom-up levels sweep all vertices (they are chosen when the frontier is
// large).  The two queues alternate: qsel picks fq.

// Per-warp staging of queue appends in shared memory, flushed in batches so a
// queue counter sees one atomicAdd per batch rather than one per warp step.
constexpr int kMStage = 256;
struct MStage {
    int* buf;
    int cnt;   // warp-uniform
};

__device__ __forceinline__ MStage m_stage() {
    __shared__ int s_mstage[kMBlock / 32][kMStage];
    MStage st;
    st.buf = s_mstage[threadIdx.x >> 5];
    st.cnt = 0;
    return st;
}

__device__ __forceinline__ void m_flush(MStage& st, int* q, unsigned long long* len) {
    if (st.cnt == 0) return;
    __syncwarp();
    unsigned long long b = 0;
    if (lane_id() == 0) b = atomicAdd(len, (unsigned long long)st.cnt);
    b = __shfl_sync(kMFull, b, 0);
    for (int i = lane_id(); i < st.cnt; i += 32) q[b + i] = st.buf[i];
    __syncwarp();
    st.cnt = 0;
}

// Final flush of a phase, every thread of the CTA calls it: the warps'
// remaining entries go out with one atomicAdd per CTA (block scan of counts).
__device__ void m_block_flush(MStage& st, int* q, unsigned long long* len) {
    __shared__ int s_wcnt[kMBlock / 32];
    __shared__ unsigned long long s_base;
    const int lane = lane_id(), wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    if (lane == 0) s_wcnt[wib] = st.cnt;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int c = lane < nwb ? s_wcnt[lane] : 0;
        const int incl = warp_inclusive_scan(c);
        const int total = __shfl_sync(kMFull, incl, 31);
        unsigned long long b = 0;
        if (lane == 0 && total) b = atomicAdd(len, (unsigned long long)total);
        if (lane < nwb) s_wcnt[lane] = incl - c;
        if (lane == 0) s_base = b;
    }
    __syncthreads();
    const unsigned long long b = s_base + (unsigned long long)s_wcnt[wib];
    for (int i = lane; i < st.cnt; i += 32) q[b + i] = st.buf[i];
    __syncwarp();
    st.cnt = 0;
}

// Stage `v` (where `want`) for queue q; all lanes call.
__device__ __forceinline__ void m_append(MStage& st, int* q, unsigned long long* len, bool want, int v) {
    const unsigned m = __ballot_sync(kMFull, want);
    if (m) {
        if (want) st.buf[st.cnt + __popc(m & lanemask_lt())] = v;
        st.cnt += __popc(m);
        if (st.cnt > kMStage - 32) m_flush(st, q, len);
    }
}

// Push lane bits along edge (v -> u); record u the first time its next mask
// becomes nonzero.  All lanes call.
__device__ __forceinline__ void ms_push(const MultiParams& p, unsigned long long f, int u, bool act, MStage& st,
                                        int* tq, unsigned long long* tlen) {
    bool first = false;
    if (act) {
        const unsigned long long nb = f & ~ldcg64(p.seen + u);
        if (nb) first = atomicOr(p.next + u, nb) == 0ull;
    }
    m_append(st, tq, tlen, first, u);
}

// Top-down push over the frontier queue (warp-balanced gather; heavy rows
// become chunk tasks processed by ms_tasks_phase after a barrier).
__device__ void ms_td_phase(const MultiParams& p, MCtrl* c, int slot, const int* fq, long long flen, int* tq,
                            unsigned long long* tlen) {
    const int lane = lane_id();
    const long long gw = m_gtid() >> 5, nw = m_gthreads() >> 5;
    MStage st = m_stage();
    // a small frontier is spread over every warp (one gather round each)
    const long long per = flen >= nw * 32 ? 32 : max(1LL, (flen + nw - 1) / nw);
    for (long long base = gw * per; base < flen; base += nw * per) {
        const long long i = base + lane;
        int v = 0;
        unsigned long long f = 0;
        long long s = 0, e = 0;
        if (lane < per && i < flen) {
            v = __ldcg(fq + i);
            f = ldcg64(p.front + v);
            if (f) {
                // v leaves the frontier here (its mask travels in registers, or
                // with its chunk tasks); nothing else reads front[v] this phase
                p.front[v] = 0ull;
                s = __ldg(p.off + v);
                e = __ldg(p.off + v + 1);
            }
        }
        const long long deg = e - s;
        const bool big = deg > p.big_deg;
        const int mydeg = big ? 0 : (int)deg;
        unsigned bm = __ballot_sync(kMFull, big);
        while (bm) {
            const int L = __ffs(bm) - 1;
            bm &= bm - 1;
            const long long bs = __shfl_sync(kMFull, s, L), be = __shfl_sync(kMFull, e, L);
            const unsigned long long bf = __shfl_sync(kMFull, f, L);
            const long long nch = (be - bs + kMChunk - 1) / kMChunk;
            unsigned long long t0 = 0;
            if (lane == 0) t0 = atomicAdd(&c->ntask[slot], (unsigned long long)nch);
            t0 = __shfl_sync(kMFull, t0, 0);
            // the row's lane mask is kept at the slot of its first chunk
            if (lane == 0 && (long long)t0 < p.task_cap) p.hubmask[t0] = bf;
            for (long long k = lane; k < nch; k += 32) {
                const long long ti = (long long)t0 + k;
                if (ti < p.task_cap) {
                    MTask t;
                    t.start = bs + k * kMChunk;
                    t.len = (int)min((long long)kMChunk, be - t.start);
                    t.v = (int)t0;
                    p.tasks[ti] = t;
                } else {
                    raise_status(&c->b, kDevOverflow);
                }
            }
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
            const bool act = k < total;
            const int u = act ? __ldg(p.cols + sj + (k - exj)) : 0;
            ms_push(p, fj, u, act, st, tq, tlen);
        }
    }
    m_block_flush(st, tq, tlen);
}

__device__ void ms_tasks_phase(const MultiParams& p, MCtrl* c, int slot, int* tq, unsigned long long* tlen) {
    const int lane = lane_id();
    const long long gw = m_gtid() >> 5, nw = m_gthreads() >> 5;
    MStage st = m_stage();
    const long long nt = min((long long)ld_relaxed64(&c->ntask[slot]), p.task_cap);
    for (long long t = gw; t < nt; t += nw) {
        const int4 raw = __ldcg(reinterpret_cast<const int4*>(p.tasks + t));
        const long long start = (long long)(unsigned)raw.x | ((long long)raw.y << 32);
        const int len = raw.z, h = raw.w;
        const unsigned long long f = ldcg64(p.hubmask + h);
        for (int k0 = 0; k0 < len; k0 += 32) {
            const int k = k0 + lane;
            const bool act = k < len;
            const int u = act ? __ldg(p.cols + start + k) : 0;
            ms_push(p, f, u, act, st, tq, tlen);
        }
    }
    m_block_flush(st, tq, tlen);
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
            const int4 x0 = __ldg(reinterpret_cast<const int4*>(p.cols_bu + a));
            const int4 x1 = __ldg(reinterpret_cast<const int4*>(p.cols_bu + a + 4));
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
                if (q < pe) x = ldcg64(p.front + __ldg(p.cols_bu + q));
                aL |= warp_or64(x);
                if ((aL & mL) == mL) break;
            }
            if (lane == L) acc = aL;
        }
        const unsigned long long nb = acc & miss;
        if (nb) p.next[u] = nb;
    }
}

// Apply over the touched vertices (after a top-down level, whose phase already
// removed the old frontier from front): seen |= next, front = next, next = 0,
// per-lane levels; counts the new frontier (n_f, m_f), the degree of vertices
// every active lane has now seen (subtracted from m_u) and which lanes found
// anything.
__device__ void ms_apply_phase(const MultiParams& p, MCtrl* c, int slot, int iter, unsigned long long active,
                               const LaneSmem& L, const int* tq, long long tlen) {
    const long long tid = m_gtid(), nth = m_gthreads();
    unsigned long long am = 0, adone = 0, found = 0;
    for (long long i = tid; i < tlen; i += nth) {
        const int v = __ldcg(tq + i);
        const unsigned long long x = ldcg64(p.next + v);
        p.next[v] = 0ull;
        const unsigned long long s = ldcg64(p.seen + v);
        p.seen[v] = s | x;
        p.front[v] = x;
        found |= x;
        const long long deg = __ldg(p.off + v + 1) - __ldg(p.off + v);
        am += (unsigned long long)deg;
        if ((s & active) != active && ((s | x) & active) == active) adone += (unsigned long long)deg;
        unsigned long long bits = x;
        while (bits) {
            const int i2 = __ffsll((long long)bits) - 1;
            bits &= bits - 1;
            L.rows[i2][v] = iter + 1 - L.start[i2];
        }
    }
    found = warp_or64(found);
    if (lane_id() == 0 && found) atomicOr(&c->found[slot], found);
    block_add4(0, am, adone, 0, nullptr, &c->accm[slot], &c->mdone[slot], nullptr);
    if (tid == 0) c->accn[slot] = (unsigned long long)tlen;
}

// Apply after a bottom-up level, over all vertices (that level swept them all
// anyway): the same updates as ms_apply_phase, old frontier bits dropped in
// the same pass, and the new frontier listed in queue nq.
__device__ void ms_apply_all_phase(const MultiParams& p, MCtrl* c, int slot, int iter, unsigned long long active,
                                   const LaneSmem& L, int* nq, unsigned long long* nlen) {
    const long long tid = m_gtid(), nth = m_gthreads();
    MStage st = m_stage();
    unsigned long long an = 0, am = 0, adone = 0, found = 0;
    for (long long base = tid - lane_id(); base < p.n; base += nth) {
        const long long v = base + lane_id();
        unsigned long long x = 0;
        if (v < p.n) {
            x = ldcg64(p.next + v);
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
            } else if (ldcg64(p.front + v)) {
                p.front[v] = 0ull;
            }
        }
        // level rows: the warp walks the lanes any of its 32 vertices gained, one
        // lane at a time, so each store instruction writes consecutive vertices of
        // one row (a lane-by-lane walk per thread would scatter every store)
        unsigned long long ub = warp_or64(x);
        while (ub) {
            const int i2 = __ffsll((long long)ub) - 1;
            ub &= ub - 1;
            if ((x >> i2) & 1ull) L.rows[i2][v] = iter + 1 - L.start[i2];
        }
        m_append(st, nq, nlen, x != 0ull, (int)v);
    }
    m_block_flush(st, nq, nlen);
    found = warp_or64(found);
    if (lane_id() == 0 && found) atomicOr(&c->found[slot], found);
    block_add4(an, am, adone, 0, &c->accn[slot], &c->accm[slot], &c->mdone[slot], nullptr);
}

// Clear the three masks and both queue counters (grid-stride).
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

// Seed lanes in `mask` at their roots (atomics: several lanes may share a
// root); a root not yet in the frontier joins the frontier queue.  Run by the
// first warp (64 lanes at most -> two rounds).
__device__ void ms_seed_phase(const MultiParams& p, unsigned long long mask, const LaneSmem& L, int* fq,
                              unsigned long long* flen) {
    if (m_gtid() >= 32) return;
    MStage st = m_stage();
    for (int i0 = 0; i0 < 64; i0 += 32) {
        const int i = i0 + lane_id();
        bool add = false;
        int r = 0;
        if ((mask >> i) & 1ull) {
            r = p.roots[i];
            atomicOr(p.seen + r, 1ull << i);
            add = atomicOr(p.front + r, 1ull << i) == 0ull;
            L.rows[i][r] = 0;
        }
        m_append(st, fq, flen, add, r);
    }
    m_flush(st, fq, flen);
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
    ms_seed_phase(p, active, L, p.q0, &c->qlen[0]);
    if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
    // level-0 statistics from the (few) distinct roots, identical in every CTA
    long long mf = 0, mu = p.nnz;
    for (int i = 0; i < 64; i++) {
        if (!((active >> i) & 1ull)) continue;
        const int r = p.roots[i];
        bool dup = false;
        for (int j = 0; j < i; j++)
            if (((active >> j) & 1ull) && p.roots[j] == r) dup = true;
        if (dup) continue;
        const long long deg = __ldg(p.off + r + 1) - __ldg(p.off + r);
        mf += deg;
        if ((ldcg64(p.seen + r) & active) == active) mu -= deg;
    }
    int prev = 0, qsel = 0;
    for (int it = 0;; it++) {
        // counters of iteration `it` accumulate in slot it % 3 and are read by
        // every CTA after the closing barrier; the slot of iteration it + 1 is
        // cleared now (its last readers passed a barrier of iteration it - 1)
        const int slot = it % 3, sfree = (it + 1) % 3;
        if (blockIdx.x == 0 && threadIdx.x == 0) c->zero_slot(sfree);
        int* fq = qsel ? p.q1 : p.q0;
        int* tq = qsel ? p.q0 : p.q1;
        const long long flen = (long long)ld_relaxed64(&c->qlen[qsel]);
        unsigned long long* tlen = &c->qlen[qsel ^ 1];
        const int dir = ms_decide(p, prev, flen, mf, mu);
        if (dir == 0) {
            ms_td_phase(p, c, slot, fq, flen, tq, tlen);
            if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            if (ld_relaxed64(&c->ntask[slot]) > 0) {
                ms_tasks_phase(p, c, slot, tq, tlen);
                if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            }
            ms_apply_phase(p, c, slot, it, active, L, tq, (long long)ld_relaxed64(tlen));
        } else {
            ms_bu_phase(p, active);
            if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            ms_apply_all_phase(p, c, slot, it, active, L, tq, tlen);
        }
        if (m_gtid() == 0) c->qlen[qsel] = 0;   // the old frontier's queue collects the next touched set
        if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
        const long long nt = (long long)ld_relaxed64(&c->accn[slot]);
        qsel ^= 1;
        if (nt == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) c->iterations = it + 1;
            break;
        }
        mu -= (long long)ld_relaxed64(&c->mdone[slot]);
        mf = (long long)ld_relaxed64(&c->accm[slot]);
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

// Clear the three masks of a slot (used when a server slot is created).
__global__ void __launch_bounds__(kMBlock) ms_clear_kernel(MultiParams p) { ms_clear_phase(p); }

// ---------------------------------------------------------------- server driver

// One launch of a server slot: optional admission of new lanes (drop the
// stale bits of `drop` lanes, fill new rows with -1, seed new roots), then
// levels iter0, iter0+1, ... for all `active` lanes until a lane's frontier
// comes back empty (its result is final), the union frontier is empty, or
// max_iters levels ran.  The direction per level follows the union frontier
// (top-down -> bottom-up when m_f * alpha > nnz / 2, back when n_f * beta < n;
// the per-lane unvisited degree m_u is not tracked when lanes start at
// different levels).  Results for the host: s_done, s_finished, s_nf, s_mf,
// s_dir in the control block (which persists across launches of the slot).
__global__ void __launch_bounds__(kMBlock, 2) bfs_serve_kernel(MultiParams p, int iter0, int max_iters,
                                                                unsigned long long newmask,
                                                                unsigned long long drop) {
    __shared__ LaneSmem L;
    load_lanes(p, L);
    MCtrl* c = p.ctrl;
    const unsigned long long active = p.active;
    const long long tid = m_gtid(), nth = m_gthreads();
    int qsel = c->s_qsel;
    if (drop) {
        // lanes being reused: remove their previous query's bits
        const unsigned long long keep = ~drop;
        for (long long v = tid; v < p.n; v += nth) {
            const unsigned long long s = p.seen[v];
            if (s & drop) p.seen[v] = s & keep;
            const unsigned long long f = p.front[v];
            if (f & drop) p.front[v] = f & keep;
        }
    }
    if (newmask | drop) {
        ms_fill_rows(p, newmask, L);
        if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
        ms_seed_phase(p, newmask, L, qsel ? p.q1 : p.q0, &c->qlen[qsel]);
        if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
    }
    long long mf = c->s_mf;
    int prev = c->s_dir;
    int it = iter0, done = 0;
    long long nt = 0;
    unsigned long long finished = 0;
    for (; done < max_iters; it++) {
        const int slot = it % 3, sfree = (it + 1) % 3;
        if (blockIdx.x == 0 && threadIdx.x == 0) c->zero_slot(sfree);
        int* fq = qsel ? p.q1 : p.q0;
        int* tq = qsel ? p.q0 : p.q1;
        const long long flen = (long long)ld_relaxed64(&c->qlen[qsel]);
        unsigned long long* tlen = &c->qlen[qsel ^ 1];
        int dir;
        if (p.mode == BFS_MODE_TD_ONLY) dir = 0;
        else if (p.mode == BFS_MODE_BU_ONLY) dir = 1;
        else if (prev == 0) dir = (mf * (long long)p.alpha > p.nnz / 2) ? 1 : 0;
        else dir = (flen * (long long)p.beta < p.n) ? 0 : 1;
        if (dir == 0) {
            ms_td_phase(p, c, slot, fq, flen, tq, tlen);
            if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            if (ld_relaxed64(&c->ntask[slot]) > 0) {
                ms_tasks_phase(p, c, slot, tq, tlen);
                if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            }
            ms_apply_phase(p, c, slot, it, active, L, tq, (long long)ld_relaxed64(tlen));
        } else {
            ms_bu_phase(p, active);
            if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            ms_apply_all_phase(p, c, slot, it, active, L, tq, tlen);
        }
        if (tid == 0) c->qlen[qsel] = 0;
        if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
        nt = (long long)ld_relaxed64(&c->accn[slot]);
        qsel ^= 1;
        done++;
        prev = dir;
        mf = (long long)ld_relaxed64(&c->accm[slot]);
        finished = active & ~ld_relaxed64(&c->found[slot]);
        if (finished || nt == 0) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->s_done = done;
        c->s_finished = finished;
        c->s_nf = nt;
        c->s_mf = mf;
        c->s_dir = prev;
        c->s_qsel = qsel;
    }
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
    w.seen = (unsigned long long*)mem_of(g, w).alloc(nb, s);
    w.front = (unsigned long long*)mem_of(g, w).alloc(nb, s);
    w.next = (unsigned long long*)mem_of(g, w).alloc(nb, s);
    w.ctrl = mem_of(g, w).alloc(sizeof(MCtrl), s);
    w.tasks = mem_of(g, w).alloc(sizeof(MTask) * (size_t)task_cap, s);
    w.hubmask = mem_of(g, w).alloc(sizeof(unsigned long long) * (size_t)task_cap, s);
    w.lanes = mem_of(g, w).alloc(sizeof(bfsk::LaneTable), s);
    w.q0 = (int*)mem_of(g, w).alloc(sizeof(int) * (size_t)(g->n + 64), s);
    w.q1 = (int*)mem_of(g, w).alloc(sizeof(int) * (size_t)(g->n + 64), s);
    w.task_cap = task_cap;
    if (!w.seen || !w.front || !w.next || !w.ctrl || !w.tasks || !w.hubmask || !w.lanes || !w.q0 || !w.q1) {
        w.ready = true;
        multi_free(g, w);
        return fail(BFS_ERR_OOM, "multi-source work buffers: device allocation failed");
    }
    w.bytes = 3 * nb + sizeof(MCtrl) + (sizeof(MTask) + 8) * (size_t)task_cap + sizeof(bfsk::LaneTable) +
              2 * sizeof(int) * (size_t)(g->n + 64);
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
    mem_of(g, w).release(w.seen, nb, nullptr);
    mem_of(g, w).release(w.front, nb, nullptr);
    mem_of(g, w).release(w.next, nb, nullptr);
    mem_of(g, w).release(w.ctrl, sizeof(MCtrl), nullptr);
    mem_of(g, w).release(w.tasks, sizeof(MTask) * (size_t)w.task_cap, nullptr);
    mem_of(g, w).release(w.hubmask, sizeof(unsigned long long) * (size_t)w.task_cap, nullptr);
    mem_of(g, w).release(w.lanes, sizeof(bfsk::LaneTable), nullptr);
    mem_of(g, w).release(w.q0, sizeof(int) * (size_t)(g->n + 64), nullptr);
    mem_of(g, w).release(w.q1, sizeof(int) * (size_t)(g->n + 64), nullptr);
    DeviceAlloc* keep = w.mem;   // the allocator choice outlives the buffers
    w = MultiWork();
    w.mem = keep;
}

bfs_status multi_prepare(bfs_graph* g, cudaStream_t s) { return multi_alloc(g, g->multi, s); }
void multi_release(bfs_graph* g) { multi_free(g, g->multi); }

static MultiParams multi_params(bfs_graph* g, MultiWork& w, const bfs_options& opt) {
    MultiParams p;
    memset(&p, 0, sizeof p);
    p.off = reinterpret_cast<const long long*>(g->offsets);
    p.cols = g->cols;
    p.cols_bu = (opt.bu_rows == BFS_BU_ROWS_HUB_FIRST && g->cols_hf) ? g->cols_hf : g->cols;
    p.n = g->n;
    p.nnz = g->nnz;
    p.seen = w.seen;
    p.front = w.front;
    p.next = w.next;
    p.ctrl = reinterpret_cast<MCtrl*>(w.ctrl);
    p.q0 = w.q0;
    p.q1 = w.q1;
    p.tasks = reinterpret_cast<MTask*>(w.tasks);
    p.hubmask = reinterpret_cast<unsigned long long*>(w.hubmask);
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
    p.expected = (unsigned)w.grid + (unsigned)(g->debug_barrier_extra > 0 ? g->debug_barrier_extra : 0);
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

// ---------------------------------------------------------------- server driver (host side)

size_t ms_lane_table_bytes() { return sizeof(bfsk::LaneTable); }

void ms_lane_table_set(void* table_host, int lane, int32_t* row, int start, int root) {
    bfsk::LaneTable* t = reinterpret_cast<bfsk::LaneTable*>(table_host);
    t->rows[lane] = row;
    t->prow[lane] = nullptr;
    t->start[lane] = start;
    t->roots[lane] = root;
}

int ms_serve_max_grid(bfs_graph* g, MultiWork& w) { (void)g; return w.grid; }

bfs_status ms_serve_reset(bfs_graph* g, MultiWork& w, cudaStream_t s) {
    bfs_options o;
    bfs_options_default(&o);
    if (g->cols_hf) o.bu_rows = BFS_BU_ROWS_HUB_FIRST;
    MultiParams p = multi_params(g, w, o);
    bfsk::ms_clear_kernel<<<w.grid, w.block, 0, s>>>(p);
    BFS_CUDA_TRY(cudaGetLastError());
    BFS_CUDA_TRY(cudaMemsetAsync(w.ctrl, 0, sizeof(MCtrl), s));
    return BFS_OK;
}

bfs_status ms_serve_launch(bfs_graph* g, MultiWork& w, const void* lane_table_host, unsigned long long newmask,
                           unsigned long long drop, unsigned long long active, int iter0, int max_iters, int grid,
                           void* ctrl_pinned, cudaStream_t s) {
    bfs_options o;
    bfs_options_default(&o);
    if (g->cols_hf) o.bu_rows = BFS_BU_ROWS_HUB_FIRST;   // levels do not depend on the row order
    MultiParams p = multi_params(g, w, o);
    p.active = active;
    grid = std::max(1, std::min(grid, w.grid));
    p.expected = (unsigned)grid;
    if (newmask)
        BFS_CUDA_TRY(cudaMemcpyAsync(w.lanes, lane_table_host, sizeof(bfsk::LaneTable), cudaMemcpyHostToDevice, s));
    // the barrier state (first member of the control block) restarts at zero for
    // every launch, as the grid size varies between launches; the rest of the
    // control block carries over
    static_assert(offsetof(MCtrl, b) == 0, "barrier state leads the control block");
    BFS_CUDA_TRY(cudaMemsetAsync(w.ctrl, 0, sizeof(bfsk::BarrierState), s));
    void* args[] = {&p, &iter0, &max_iters, &newmask, &drop};
    BFS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)bfsk::bfs_serve_kernel, dim3(grid), dim3(w.block), args, 0, s));
    BFS_CUDA_TRY(cudaMemcpyAsync(ctrl_pinned, w.ctrl, sizeof(MCtrl), cudaMemcpyDeviceToHost, s));
    return BFS_OK;
}

}  // namespace bfsrt
