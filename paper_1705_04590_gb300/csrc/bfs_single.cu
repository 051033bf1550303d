// bfs_single.cu -- single-source (and multi-root) direction-optimizing BFS as
// one persistent cooperative launch per search.
//
// The level loop of Algorithm 1/2 runs entirely on the device: every CTA
// evaluates the direction rule of "Parallel Direction-Optimizing BFS" from
// the same device counters, does its share of the level, and meets the
// others at a bounded grid barrier.  No host round trip happens per level.
//
// Level d (frontier F_d, n_f = |F_d|, m_f = sum of degrees over F_d, m_u =
// degree sum of the vertices not yet reached):
//   direction: top-down -> bottom-up when m_f * alpha > m_u,
//              bottom-up -> top-down when n_f * beta < n.
//   top-down  (Algorithm 1 inner loops; the local discovery of Algorithm 3):
//              for u in the queue, for v in adj(u): claim v by an atomicOr on
//              the visited bitmap; the winner writes parent/level and appends
//              v to the next queue (warp ballot + one atomicAdd per warp).
//              Frontier vertices of degree > big_deg are cut into edge chunks
//              that all warps share after a barrier (load balance on R-MAT
//              hubs); the rest are gathered warp-cooperatively (a warp prefix
//              sum over its 32 vertices' degrees maps lanes onto edges).
//   bottom-up (Algorithm 2 inner loops; the local search of Algorithm 4):
//              a warp owns 32 consecutive vertices (one word of the
//              completed bitmap c); each unvisited lane scans its sorted row
//              in 16-byte (int4) pieces, testing frontier-bitmap bits, and
//              stops at the first hit; long rows continue warp-cooperatively.
//              Found vertices are written to the next-frontier bitmap as one
//              ballot word per warp (no atomics: the warp owns the word).
//   conversion: queue -> bitmap before a bottom-up level that follows a
//              top-down one, bitmap -> queue (popcount + warp scan) before a
//              top-down level that follows a bottom-up one.
// Membership tests read only the current frontier; next is separate and
// swapped in after the level (the reading of Algorithm 2 that keeps levels
// exact).
#include <climits>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "bfs_common.cuh"
#include "bfs_internal.h"

namespace bfsk {

#ifndef BFS_BLOCK
#define BFS_BLOCK 512
#endif
constexpr int kBlock = BFS_BLOCK;  // CSR kernel
constexpr int kDBlock = 1024;   // DCSC kernel (one CTA per vertex block)
constexpr int kWarps = 32;      // shared-memory per-warp arrays sized for up to 1024 threads
constexpr int kChunk = 256;    // edges per top-down chunk task of the allocation-free entry point
constexpr int kDefaultChunk = 128;   // default of options.td_chunk (measured best at R-MAT 26)
constexpr int kMinChunk = 64;  // smallest chunk task: the task lists are sized for it
constexpr int kStage = 256;    // per-warp shared-memory staging of next-queue entries

// Shared memory that phases of the CSR kernel borrow in turn: the top-down
// staging slices, and bottom-up phase A's searcher lists, whose two halves are
// the frontier buffers of the cluster levels.
__shared__ __align__(16) int g_stage[kBlock / 32][kStage];
__shared__ __align__(16) int g_stage_d[kDBlock / 32][kStage];   // the DCSC kernel's (more warps per CTA)
__shared__ __align__(16) unsigned short g_list[kBlock / 32][1024];
constexpr long long kPrefetchNf = 1 << 16;   // top-down levels below this prefetch the next rows
#ifndef BFS_TD_CHECK
#define BFS_TD_CHECK 0   // 1: top-down gather reads the visited word before claiming (hub chunks always do)
#endif
#ifndef BFS_MIN_BLOCKS
#define BFS_MIN_BLOCKS 2
#endif
constexpr unsigned kFull = 0xffffffffu;
constexpr size_t kSingleDynSmem = 0;   // the CSR kernel uses static shared memory only

struct Task {
    long long start;
    int len;
    int u;
};

struct SingleParams {
    const long long* __restrict__ off;
    const int* __restrict__ cols;
    const int* __restrict__ cols_bu;     // rows as the bottom-up steps scan them (cols, or hub-first)
    // heads of the hub-first rows: heads[8u .. 8u+7] = {deg(u), r0 .. r6}, 32-byte aligned
    const int* __restrict__ heads;
    // first[u] = r0 | (deg(u) >= 2) << 31: the first id of u's hub-first row and
    // whether the row goes on (null: bottom-up scans the rows from their
    // offsets); a bottom-up level over the hub-first rows streams it in vertex
    // order
    const int* __restrict__ first;
    const unsigned char* __restrict__ deg8;   // min(deg(u), 255); null: degrees from the offsets
    // the rows bottom-up steps scan: cols_bu with these offsets (off itself, or on a
    // directed graph the transpose's: the in-edge rows)
    const long long* __restrict__ off_bu;
    const unsigned char* __restrict__ deg8_in;   // directed: min(in-degree, 255)
    int directed;     // 1: off/cols are out-edge rows, off_bu/cols_bu in-edge rows
    const unsigned* __restrict__ isolated;
    long long n, nnz, W;
    int* parent;
    int* level;
    // level staging: one byte per vertex during the search (kLvUnseen / depth /
    // kLvDeep); after the last level a final pass writes `level` and `parent` in
    // whole sectors from it.  null = write `level` and `parent` directly over a
    // -1 fill
    unsigned char* lv8;
    // with lv8: bit v set when v's parent is first[v] (a bottom-up hit on the
    // first probe), so that no parent store is made for it during the search
    unsigned* pfirst;
    unsigned* visited;
    unsigned* front0;
    unsigned* front1;
    int* queue0;
    int* queue1;
    Task* tasks;
    long long task_cap;
    Ctrl* ctrl;
    bfs_level_record* rec;
    int rec_cap;
    int root0;     // the root when nroots == 1
    int nroots;    // > 1: roots already copied into queue0[0..nroots)
    int mode, alpha, beta, parent_mode, big_deg;
    int td_chunk;      // edges per top-down chunk task (>= kMinChunk)
    // cluster levels: CTAs per thread-block cluster of the launch (1 = none);
    // cluster 0 runs a top-down level alone while the frontier holds at most
    // clu_nf vertices and clu_mf edges and no vertex of degree above clu_big
    // (0 when off: the top-down flushes then count no heavy vertices)
    int clu_c, clu_big;
    long long clu_nf, clu_mf;
    unsigned long long seed;
    unsigned long long timeout_ns;
    unsigned expected;
    // DCSC tiles (layout BFS_LAYOUT_DCSC_TILED)
    const long long* __restrict__ tile_ptr;
    const int* __restrict__ jc;
    const long long* __restrict__ cp;
    const int* __restrict__ ir;
    int nb;            // p blocks
    long long B;       // vertices per block (multiple of 32)
    long long Bw;      // words per block
};

constexpr int TD = 0, BU = 1;

__device__ __forceinline__ int decide_dir(const SingleParams& p, int prev, long long nf, long long mf,
                                          long long mu, int d) {
    switch (p.mode) {
        case BFS_MODE_TD_ONLY: return TD;
        case BFS_MODE_BU_ONLY: return BU;
        case BFS_MODE_RANDOM:
            return (int)(mix64(p.seed + 0x9E3779B97F4A7C15ULL * (unsigned long long)(d + 1)) >> 63);
        default:
            if (prev == TD) return (mf * (long long)p.alpha > mu) ? BU : TD;
            return (nf * (long long)p.beta < p.n) ? TD : BU;
    }
}

#ifndef BFS_BU_WIN
#define BFS_BU_WIN 8     // ids in the first bottom-up window: 4 (one int4) or 8 (two)
#endif
constexpr int kWin = BFS_BU_WIN;
static_assert(kWin == 4 || kWin == 8, "window is one or two int4");

#ifndef BFS_EVICT
#define BFS_EVICT 1      // 1: bottom-up graph reads marked evict-first in L2
#endif

// Bottom-up reads of the graph stream through L2 once per level; marking them
// evict-first leaves L2 to the bitmaps and the output sectors being filled.
#if BFS_EVICT
__device__ __forceinline__ unsigned long long evict_first_policy() {
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
#endif

__device__ __forceinline__ int4 ld_stream4(const int4* a) {
#if BFS_EVICT
    int4 v;
    asm("ld.global.nc.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(a), "l"(evict_first_policy()));
    return v;
#else
    return __ldg(a);
#endif
}

// one 32-byte record (a 256-bit load; the address is 32-byte aligned)
__device__ __forceinline__ void ld_stream8(const int* a, int4& lo, int4& hi) {
#if BFS_EVICT
    asm("ld.global.nc.L2::cache_hint.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8], %9;"
        : "=r"(lo.x), "=r"(lo.y), "=r"(lo.z), "=r"(lo.w), "=r"(hi.x), "=r"(hi.y), "=r"(hi.z), "=r"(hi.w)
        : "l"(a), "l"(evict_first_policy()));
#else
    asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(lo.x), "=r"(lo.y), "=r"(lo.z), "=r"(lo.w), "=r"(hi.x), "=r"(hi.y), "=r"(hi.z), "=r"(hi.w)
        : "l"(a));
#endif
}

__device__ __forceinline__ int ld_stream32(const int* a) {
#if BFS_EVICT
    int v;
    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(evict_first_policy()));
    return v;
#else
    return __ldg(a);
#endif
}

__device__ __forceinline__ unsigned ld_stream_u8(const unsigned char* a) {
#if BFS_EVICT
    unsigned short v;
    asm("ld.global.nc.L2::cache_hint.u8 %0, [%1], %2;" : "=h"(v) : "l"(a), "l"(evict_first_policy()));
    return v;
#else
    return __ldg(a);
#endif
}

__device__ __forceinline__ long long ld_stream64(const long long* a) {
#if BFS_EVICT
    long long v;
    asm("ld.global.nc.L2::cache_hint.s64 %0, [%1], %2;" : "=l"(v) : "l"(a), "l"(evict_first_policy()));
    return v;
#else
    return __ldg(a);
#endif
}

// row u's bounds [s, e) in the column array
__device__ __forceinline__ void row_of(const SingleParams& p, int u, long long& s, long long& e) {
    s = __ldg(p.off + u);
    e = __ldg(p.off + u + 1);
}

// row u of the rows bottom-up steps scan (cols_bu)
__device__ __forceinline__ void bu_row_of(const SingleParams& p, int u, long long& s, long long& e) {
    s = __ldg(p.off_bu + u);
    e = __ldg(p.off_bu + u + 1);
}

__device__ __forceinline__ void bu_row_of_stream(const SingleParams& p, int u, long long& s, long long& e) {
    s = ld_stream64(p.off_bu + u);
    e = ld_stream64(p.off_bu + u + 1);
}

__device__ __forceinline__ long long deg_of(const SingleParams& p, int u) {
    long long s, e;
    row_of(p, u, s, e);
    return e - s;
}

// deg(u) given its byte d8 = min(deg(u), 255): the offsets only for 255
__device__ __forceinline__ long long deg_from8(const SingleParams& p, int u, unsigned d8) {
    return d8 < 255u ? (long long)d8 : deg_of(p, u);
}

constexpr unsigned char kLvUnseen = 255;   // not reached (yet)
constexpr unsigned char kLvDeep = 254;     // depth >= 254: the int32 level holds it

__device__ __forceinline__ void set_level(const SingleParams& p, int v, int lev) {
    if (p.lv8) {
        if (lev < kLvDeep) {
            p.lv8[v] = (unsigned char)lev;
            return;
        }
        p.lv8[v] = kLvDeep;
    }
    if (p.level) p.level[v] = lev;
}

// level of u as far as the search has got (-1 = not reached), for readers inside the launch
__device__ __forceinline__ int get_level(const SingleParams& p, int u) {
    if (p.lv8) {
        const unsigned b = __ldcg(p.lv8 + u);
        if (b == kLvUnseen) return -1;
        if (b != kLvDeep) return (int)b;
    }
    return __ldcg(p.level + u);
}

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gthreads() { return (long long)gridDim.x * blockDim.x; }

// Fill a[0..n) with -1, using 16-byte stores for the aligned body.
__device__ void fill_minus_one(int* a, long long n) {
    const long long tid = gtid(), nth = gthreads();
    const long long head = ((16 - ((unsigned long long)a & 15)) & 15) / 4;
    const long long h = head < n ? head : n;
    if (tid < h) a[tid] = -1;
    const long long body = (n - h) / 4;
    int4* v = reinterpret_cast<int4*>(a + h);
    const int4 m1 = make_int4(-1, -1, -1, -1);
    for (long long i = tid; i < body; i += nth) v[i] = m1;
    for (long long i = h + body * 4 + tid; i < n; i += nth) a[i] = -1;
}

// parent/level fill, completed bitmap = isolated vertices (+ root), clear both
// frontier bitmaps.  The root's own entries are written after the barrier
// that ends this phase.
// lv8 is 16-byte aligned (work buffer)
__device__ void fill_bytes(unsigned char* a, long long n, unsigned char b) {
    const long long tid = gtid(), nth = gthreads();
    const unsigned w = 0x01010101u * b;
    const uint4 v4 = make_uint4(w, w, w, w);
    const long long body = n / 16;
    for (long long i = tid; i < body; i += nth) reinterpret_cast<uint4*>(a)[i] = v4;
    for (long long i = body * 16 + tid; i < n; i += nth) a[i] = b;
}

// After the last level: the outputs in whole sectors, 8 vertices (one 32-byte
// sector of each output) per thread.  level[v] = the staged byte (kLvUnseen ->
// -1); vertices at depth >= 254 already hold their int32 level and are left
// alone.  parent[v] = -1 when v was not reached, first[v] when its pfirst bit is
// set (found bottom-up on its first probe), else the value written during the
// search (the root, a top-down claim, a later bottom-up probe), read back so
// that the sector is still written whole: a partial-sector store costs a read
// of the sector from DRAM anyway.
__device__ void materialise(const SingleParams& p) {
    const long long tid = gtid(), nth = gthreads();
    const long long groups = (p.n + 7) / 8;
    const bool lvec = p.level && (((unsigned long long)p.level & 15) == 0);
    const bool pvec = p.parent && (((unsigned long long)p.parent & 15) == 0);
    for (long long gi = tid; gi < groups; gi += nth) {
        const long long v0 = gi * 8;
        const bool full = v0 + 8 <= p.n;
        const unsigned valid = full ? 0xFFu : ((1u << (unsigned)(p.n - v0)) - 1u);
        const uint2 lb = __ldcg(reinterpret_cast<const uint2*>(p.lv8 + v0));
        // most sectors hold a first-probe hit: load its plane values together with
        // the staged bytes instead of after them
        int4 fa = make_int4(-1, -1, -1, -1), fb = fa;
        if (p.parent && p.pfirst && p.first) {
            fa = ld_stream4(reinterpret_cast<const int4*>(p.first + v0));
            fb = ld_stream4(reinterpret_cast<const int4*>(p.first + v0) + 1);
        }
        unsigned reached = 0, deep = 0;
        int lv[8];
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const unsigned b = ((k < 4 ? lb.x : lb.y) >> (8 * (k & 3))) & 0xFFu;
            lv[k] = b == kLvUnseen ? -1 : (int)b;
            if (b != kLvUnseen) reached |= 1u << k;
            if (b == kLvDeep) deep |= 1u << k;
        }
        reached &= valid;
        if (p.level) {
            if (lvec && full && !deep) {
                int4* o = reinterpret_cast<int4*>(p.level + v0);
                o[0] = make_int4(lv[0], lv[1], lv[2], lv[3]);
                o[1] = make_int4(lv[4], lv[5], lv[6], lv[7]);
            } else {
#pragma unroll
                for (int k = 0; k < 8; k++)
                    if (((valid & ~deep) >> k) & 1u) p.level[v0 + k] = lv[k];
            }
        }
        if (p.parent) {
            const unsigned pf = p.pfirst ? ((__ldcg(p.pfirst + (v0 >> 5)) >> (v0 & 31)) & reached) : 0u;
            const unsigned direct = reached & ~pf;
            int f[8], q[8];
#pragma unroll
            for (int k = 0; k < 8; k++) f[k] = q[k] = -1;
            if (pf) {
                const int m = 0x7FFFFFFF;   // bit 31 flags a row that goes on
                f[0] = fa.x & m; f[1] = fa.y & m; f[2] = fa.z & m; f[3] = fa.w & m;
                f[4] = fb.x & m; f[5] = fb.y & m; f[6] = fb.z & m; f[7] = fb.w & m;
            }
            if (direct) {
                if (pvec && full) {
                    const int4 a = __ldcg(reinterpret_cast<const int4*>(p.parent + v0));
                    const int4 b = __ldcg(reinterpret_cast<const int4*>(p.parent + v0) + 1);
                    q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w;
                    q[4] = b.x; q[5] = b.y; q[6] = b.z; q[7] = b.w;
                } else {
#pragma unroll
                    for (int k = 0; k < 8; k++)
                        if ((direct >> k) & 1u) q[k] = __ldcg(p.parent + v0 + k);
                }
            }
            int o[8];
#pragma unroll
            for (int k = 0; k < 8; k++) o[k] = !((reached >> k) & 1u) ? -1 : ((pf >> k) & 1u) ? f[k] : q[k];
            if (pvec && full) {
                int4* po = reinterpret_cast<int4*>(p.parent + v0);
                po[0] = make_int4(o[0], o[1], o[2], o[3]);
                po[1] = make_int4(o[4], o[5], o[6], o[7]);
            } else {
#pragma unroll
                for (int k = 0; k < 8; k++)
                    if ((valid >> k) & 1u) p.parent[v0 + k] = o[k];
            }
        }
    }
}

__device__ void init_phase(const SingleParams& p) {
    const long long tid = gtid(), nth = gthreads();
    const bool single = p.nroots == 1;
    const long long r = p.root0;
    if (p.lv8) {
        // the outputs are written once, by the final pass
        fill_bytes(p.lv8, p.n, kLvUnseen);
    } else {
        if (p.parent) fill_minus_one(p.parent, p.n);
        if (p.level) fill_minus_one(p.level, p.n);
    }
    const long long rw = single ? (r >> 5) : -1;
    const unsigned rb = single ? (1u << (r & 31)) : 0u;
    for (long long w = tid; w < p.W; w += nth) {
        unsigned x = __ldg(p.isolated + w);
        if (w == rw) x |= rb;
        p.visited[w] = x;
        p.front0[w] = 0u;
        p.front1[w] = 0u;
        if (p.pfirst) p.pfirst[w] = 0u;
    }
    if (single && tid == 0) {
        p.queue0[0] = (int)r;
        p.ctrl->tail[0] = 1ull;
        p.ctrl->accm[0] = (unsigned long long)deg_of(p, r);
    }
}

// multi-root seeding (after the fill): roots already sit in queue0.
__device__ void seed_roots_phase(const SingleParams& p) {
    const long long tid = gtid(), nth = gthreads();
    unsigned long long m = 0, mi = 0;
    for (long long i = tid; i < p.nroots; i += nth) {
        const int r = __ldcg(p.queue0 + i);
        atomicOr(p.visited + (r >> 5), 1u << (r & 31));
        if (p.parent) p.parent[r] = r;
        set_level(p, r, 0);
        m += (unsigned long long)deg_of(p, r);
        if (p.directed) {
            long long s, e;
            bu_row_of(p, r, s, e);
            mi += (unsigned long long)(e - s);
        }
    }
    block_add4(m, mi, 0, 0, &p.ctrl->accm[0], &p.ctrl->dsum_in[0], nullptr, nullptr);
    if (tid == 0) p.ctrl->tail[0] = (unsigned long long)p.nroots;
}

// ------------------------------------------------------------------ top-down

// Per-warp staging of next-queue entries in shared memory, flushed to the
// global queue in batches: the queue tail sees one atomicAdd per batch
// instead of one per warp iteration with a claim.
struct WarpStage {
    int* buf;   // kStage entries of this warp's shared-memory slice
    int cnt;    // warp-uniform fill level
    bool pf;    // prefetch the rows of flushed vertices into L2 (small levels)
    bool nodeg;    // no degrees at the flush (a directed graph sums them after the level)
    unsigned hv;   // this lane's flushed vertices of degree above the cluster-level cap
};

// Degree of a vertex just appended to the next queue, into acc_m.  On small
// levels the next level is latency-bound: start its column reads now.
__device__ __forceinline__ void flush_degree(const SingleParams& p, int v, bool pf, unsigned long long& acc_m,
                                             unsigned& hv) {
    const unsigned d8 = p.deg8 ? (unsigned)__ldg(p.deg8 + v) : 255u;
    if (d8 < 255u && !pf) {
        acc_m += d8;
        hv += (int)d8 > p.clu_big;
        return;
    }
    long long rs, re;
    row_of(p, v, rs, re);
    acc_m += (unsigned long long)(re - rs);
    hv += re - rs > (long long)p.clu_big;
    if (pf && re > rs) asm volatile("prefetch.global.L2 [%0];" ::"l"(p.cols + rs));
}

// Write st.buf[0..cnt) to qnext[base..] and add their degrees (the next
// frontier's m_f, read here in batches rather than on the claim path) to acc_m:
// a lane takes up to kFlushBatch entries per step and has all their degree bytes
// in flight together (one by one they would be a chain of dependent DRAM reads).
constexpr int kFlushBatch = 8;

__device__ __forceinline__ void flush_entries(const SingleParams& p, WarpStage& st, int* qnext,
                                              unsigned long long base, unsigned long long& acc_m) {
    const int lane = lane_id();
    if (st.nodeg) {
        for (int i = lane; i < st.cnt; i += 32) qnext[base + i] = st.buf[i];
        return;
    }
    if (!p.deg8 || st.pf) {
        for (int i = lane; i < st.cnt; i += 32) {
            const int v = st.buf[i];
            qnext[base + i] = v;
            flush_degree(p, v, st.pf, acc_m, st.hv);
        }
        return;
    }
    for (int i0 = 0; i0 < st.cnt; i0 += 32 * kFlushBatch) {
        unsigned d8[kFlushBatch];
        int vs[kFlushBatch];
#pragma unroll
        for (int k = 0; k < kFlushBatch; k++) {
            const int i = i0 + k * 32 + lane;
            vs[k] = i < st.cnt ? st.buf[i] : -1;
            d8[k] = vs[k] >= 0 ? (unsigned)__ldg(p.deg8 + vs[k]) : 0u;
        }
#pragma unroll
        for (int k = 0; k < kFlushBatch; k++) {
            if (vs[k] < 0) continue;
            qnext[base + i0 + k * 32 + lane] = vs[k];
            const long long dg = d8[k] < 255u ? (long long)d8[k] : deg_of(p, vs[k]);
            acc_m += (unsigned long long)dg;
            st.hv += dg > (long long)p.clu_big;
        }
    }
}

__device__ __forceinline__ void stage_flush(const SingleParams& p, WarpStage& st, int* qnext,
                                            unsigned long long* tail, unsigned long long& acc_m) {
    if (st.cnt == 0) return;
    __syncwarp();
    unsigned long long base = 0;
    if (lane_id() == 0) base = atomicAdd(tail, (unsigned long long)st.cnt);
    base = __shfl_sync(kFull, base, 0);
    flush_entries(p, st, qnext, base, acc_m);
    __syncwarp();
    st.cnt = 0;
}

// End of a top-down phase: every warp's remaining staged entries are appended
// with one atomicAdd per CTA (a block scan of the warps' counts).  On small
// levels most warps hold a few entries each, and one queue-tail atomic per
// warp would serialise thousands of arrivals on one word.  All threads call.
__device__ void block_flush(const SingleParams& p, WarpStage& st, int* qnext, unsigned long long* tail,
                            unsigned long long& acc_m) {
    __shared__ int s_wcnt[kWarps];
    __shared__ unsigned long long s_bbase;
    const int lane = lane_id(), wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    if (lane == 0) s_wcnt[wib] = st.cnt;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int c = lane < nwb ? s_wcnt[lane] : 0;
        const int incl = warp_inclusive_scan(c);
        const int total = __shfl_sync(kFull, incl, 31);
        unsigned long long b = 0;
        if (lane == 0 && total) b = atomicAdd(tail, (unsigned long long)total);
        if (lane < nwb) s_wcnt[lane] = incl - c;
        if (lane == 0) s_bbase = b;
    }
    __syncthreads();
    const unsigned long long base = s_bbase + (unsigned long long)s_wcnt[wib];
    flush_entries(p, st, qnext, base, acc_m);
    __syncwarp();
    st.cnt = 0;
}

// Record the claims of one warp step: winners write parent/level and stage v.
__device__ __forceinline__ void td_stage(const SingleParams& p, int d, int u, int v, bool claimed, WarpStage& st,
                                         int* qnext, unsigned long long* tail, unsigned long long& acc_m) {
    const unsigned cm = __ballot_sync(kFull, claimed);
    if (cm) {
        if (claimed) {
            st.buf[st.cnt + __popc(cm & lanemask_lt())] = v;
            if (p.parent) p.parent[v] = u;
            set_level(p, v, d + 1);
        }
        st.cnt += __popc(cm);
        if (st.cnt > kStage - 32) stage_flush(p, st, qnext, tail, acc_m);
    }
}

// Visit edge (u, v) for the whole warp (every lane calls; `act` masks): claim
// v with an atomicOr on the visited bitmap; the winner records parent/level
// and stages v for the next queue.
__device__ __forceinline__ void td_visit(const SingleParams& p, int d, int u, int v, bool act, WarpStage& st,
                                         int* qnext, unsigned long long* tail, unsigned long long& acc_m) {
    bool claimed = false;
    if (act) {
        const unsigned bit = 1u << (v & 31);
        unsigned* wp = p.visited + (v >> 5);
        // read before claiming: most edges of a dense level meet vertices already
        // taken, and a plain L2 read does not serialise on a popular word the way
        // an atomic does
#if BFS_TD_CHECK
        if (!(__ldcg(wp) & bit)) claimed = !(atomicOr(wp, bit) & bit);
#else
        claimed = !(atomicOr(wp, bit) & bit);
#endif
    }
    td_stage(p, d, u, v, claimed, st, qnext, tail, acc_m);
}

__device__ __forceinline__ WarpStage warp_stage_in(int* buf) {
    WarpStage st;
    st.buf = buf;
    st.cnt = 0;
    st.pf = false;
    st.nodeg = false;
    st.hv = 0;
    return st;
}
// the CSR kernel's phases (kBlock threads) and the DCSC kernel's (kDBlock threads)
__device__ __forceinline__ WarpStage warp_stage() { return warp_stage_in(g_stage[threadIdx.x >> 5]); }
__device__ __forceinline__ WarpStage warp_stage_dcsc() { return warp_stage_in(g_stage_d[threadIdx.x >> 5]); }

__device__ void td_phase(const SingleParams& p, int d, const int* qcur, long long nf, int* qnext, int snext,
                         bool nodeg, unsigned long long& acc_m, unsigned long long& acc_h) {
    const int lane = lane_id();
    const long long gw = gtid() >> 5, nw = gthreads() >> 5;
    unsigned long long* tail = &p.ctrl->tail[snext];
    WarpStage st = warp_stage();
    st.nodeg = nodeg;
    st.pf = !nodeg && nf < kPrefetchNf;
    // A small frontier is spread over every warp (fewer vertices per warp, so
    // each warp's edges take one gather round instead of several dependent ones).
    const long long per = nf >= nw * 32 ? 32 : max(1LL, (nf + nw - 1) / nw);
    for (long long base = gw * per; base < nf; base += nw * per) {
        const long long i = base + lane;
        int u = 0;
        long long s = 0, e = 0;
        if (lane < per && i < nf) {
            u = __ldcg(qcur + i);
            row_of(p, u, s, e);
        }
        const long long deg = e - s;
        const bool big = deg > p.big_deg;
        const int mydeg = big ? 0 : (int)deg;
        // heavy rows become edge-chunk tasks; the warp writes each row's chunk
        // descriptors together
        unsigned bm = __ballot_sync(kFull, big);
        while (bm) {
            const int L = __ffs(bm) - 1;
            bm &= bm - 1;
            const long long bs = __shfl_sync(kFull, s, L), be = __shfl_sync(kFull, e, L);
            const int bu = __shfl_sync(kFull, u, L);
            const long long nch = (be - bs + p.td_chunk - 1) / p.td_chunk;
            unsigned long long t0 = 0;
            if (lane == 0) t0 = atomicAdd(&p.ctrl->ntask[snext], (unsigned long long)nch);
            t0 = __shfl_sync(kFull, t0, 0);
            for (long long c = lane; c < nch; c += 32) {
                const long long ti = (long long)t0 + c;
                if (ti < p.task_cap) {
                    Task t;
                    t.start = bs + c * p.td_chunk;
                    t.len = (int)min((long long)p.td_chunk, be - t.start);
                    t.u = bu;
                    p.tasks[ti] = t;
                } else {
                    raise_status(&p.ctrl->b, kDevOverflow);
                }
            }
        }
        const int incl = warp_inclusive_scan(mydeg);
        const int total = __shfl_sync(kFull, incl, 31);
        const int excl = incl - mydeg;
        for (int k0 = 0; k0 < total; k0 += 32) {
            const int k = k0 + lane;
            int j = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int c = __shfl_sync(kFull, incl, j + step - 1);
                if (c <= k) j += step;
            }
            const long long sj = __shfl_sync(kFull, s, j);
            const int exj = __shfl_sync(kFull, excl, j);
            const int uj = __shfl_sync(kFull, u, j);
            const bool act = k < total;
            const int v = act ? __ldg(p.cols + sj + (k - exj)) : 0;
            td_visit(p, d, uj, v, act, st, qnext, tail, acc_m);
        }
    }
    block_flush(p, st, qnext, tail, acc_m);
    acc_h += st.hv;
}

__device__ void task_phase(const SingleParams& p, int d, long long ntask, int* qnext, int snext, bool nodeg,
                           unsigned long long& acc_m, unsigned long long& acc_h) {
    const int lane = lane_id();
    const long long gw = gtid() >> 5, nw = gthreads() >> 5;
    unsigned long long* tail = &p.ctrl->tail[snext];
    WarpStage st = warp_stage();
    st.nodeg = nodeg;
    const long long nt = ntask < p.task_cap ? ntask : p.task_cap;
    for (long long t = gw; t < nt; t += nw) {
        const int4 raw = __ldcg(reinterpret_cast<const int4*>(p.tasks + t));
        const long long start = (long long)(unsigned)raw.x | ((long long)raw.y << 32);
        const int len = raw.z, u = raw.w;
        // four independent edges per lane per step (coalesced across the warp)
        for (int k0 = 0; k0 < len; k0 += 128) {
            int v[4];
            bool act[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int k = k0 + q * 32 + lane;
                act[q] = k < len;
                v[q] = act[q] ? __ldg(p.cols + start + k) : 0;
            }
            // all four reads in flight, then all four claims, then the staging
            unsigned seen[4];
#pragma unroll
            for (int q = 0; q < 4; q++) seen[q] = act[q] ? __ldcg(p.visited + (v[q] >> 5)) : kFull;
            bool claimed[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const unsigned bit = 1u << (v[q] & 31);
                if (!(seen[q] & bit)) seen[q] = atomicOr(p.visited + (v[q] >> 5), bit);
                else seen[q] = bit;
            }
#pragma unroll
            for (int q = 0; q < 4; q++) claimed[q] = act[q] && !(seen[q] & (1u << (v[q] & 31)));
#pragma unroll
            for (int q = 0; q < 4; q++) td_stage(p, d, u, v[q], claimed[q], st, qnext, tail, acc_m);
        }
    }
    block_flush(p, st, qnext, tail, acc_m);
    acc_h += st.hv;
}

// parent_mode MIN_ID, after the last level: every reached v other than a root
// takes the smallest neighbour one level closer, min{u in adj(v) : level(u) =
// level(v) - 1} (on a directed graph the smallest u with u -> v; the (select2nd,
// min) semiring of the top-down local discovery; rows are sorted, so the first
// such u in the row).  Bottom-up levels over the
// id-ordered rows already found exactly that parent; top-down claims did not.
// One pass after the loop instead of one per top-down level keeps the level
// loop's register budget free of it.
__device__ void min_parent_pass(const SingleParams& p) {
    const long long tid = gtid(), nth = gthreads();
    for (long long v = tid; v < p.n; v += nth) {
        const int lv = get_level(p, (int)v);
        if (lv <= 0) continue;
        long long s, e;
        bu_row_of(p, (int)v, s, e);   // the neighbours (in-neighbours of a directed graph), id order
        for (long long k = s; k < e; k++) {
            const int u = __ldg(p.cols_bu + k);
            if (get_level(p, u) == lv - 1) {
                p.parent[v] = u;
                break;
            }
        }
    }
}

// A directed graph's new frontier, after its level: the sum of its out-degrees
// (m_f of the direction rule) and of its in-degrees (what m_u, the in-degree
// sum of the unreached vertices, loses).  The frontier is the queue q[0..nq)
// after a top-down level (q non-null), else the bitmap f.
__device__ __forceinline__ long long out_degree(const SingleParams& p, int v) {
    const unsigned d8 = __ldg(p.deg8 + v);
    return d8 < 255u ? (long long)d8 : deg_of(p, v);
}

__device__ __forceinline__ long long in_degree(const SingleParams& p, int v) {
    const unsigned d8 = __ldg(p.deg8_in + v);
    if (d8 < 255u) return (long long)d8;
    long long s, e;
    bu_row_of(p, v, s, e);
    return e - s;
}

__device__ void frontier_degree_sums(const SingleParams& p, const int* q, long long nq, const unsigned* f,
                                     unsigned long long& sum_out, unsigned long long& sum_in) {
    const long long tid = gtid(), nth = gthreads();
    if (q) {
        for (long long i = tid; i < nq; i += nth) {
            const int v = __ldcg(q + i);
            sum_out += (unsigned long long)out_degree(p, v);
            sum_in += (unsigned long long)in_degree(p, v);
        }
    } else {
        for (long long w = tid; w < p.W; w += nth) {
            unsigned x = __ldcg(f + w);
            while (x) {
                const int v = (int)(w * 32 + __ffs(x) - 1);
                x &= x - 1;
                sum_out += (unsigned long long)out_degree(p, v);
                sum_in += (unsigned long long)in_degree(p, v);
            }
        }
    }
}

// ------------------------------------------------------------------ conversions

__device__ void queue_to_bitmap(const SingleParams& p, const int* q, long long nf, unsigned* f) {
    const long long tid = gtid(), nth = gthreads();
    for (long long i = tid; i < nf; i += nth) {
        const int v = __ldcg(q + i);
        atomicOr(f + (v >> 5), 1u << (v & 31));
    }
}

// Read-and-clear `f` into queue q (cursor *tail), clear `other` too, so both
// frontier bitmaps are zero for a later queue -> bitmap conversion.  Each
// thread takes kB2QWords consecutive words per round (two 16-byte loads), so a
// whole bitmap takes a round or two instead of one round per word per thread.
constexpr int kB2QWords = 8;

__device__ void bitmap_to_queue(const SingleParams& p, unsigned* f, unsigned* other, int* q,
                                unsigned long long* tail) {
    // rounds that are uniform across the CTA: per round the CTA claims its queue
    // range with one atomicAdd (a block scan of its threads' counts)
    __shared__ int s_wtot[kWarps];
    __shared__ unsigned long long s_qb;
    const int lane = lane_id(), wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    const long long span = (long long)gthreads() * kB2QWords;
    const bool vec = (p.W % 4) == 0;   // whole 16-byte groups (bitmaps are 16-byte aligned)
    for (long long r0 = (long long)blockIdx.x * blockDim.x * kB2QWords; r0 < p.W; r0 += span) {
        const long long w0 = r0 + (long long)threadIdx.x * kB2QWords;
        unsigned x[kB2QWords];
        if (vec && w0 + kB2QWords <= p.W) {
            const uint4 a = __ldcg(reinterpret_cast<const uint4*>(f + w0));
            const uint4 b = __ldcg(reinterpret_cast<const uint4*>(f + w0) + 1);
            x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w; x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
            const uint4 z = make_uint4(0u, 0u, 0u, 0u);
            reinterpret_cast<uint4*>(f + w0)[0] = z;
            reinterpret_cast<uint4*>(f + w0)[1] = z;
            reinterpret_cast<uint4*>(other + w0)[0] = z;
            reinterpret_cast<uint4*>(other + w0)[1] = z;
        } else {
#pragma unroll
            for (int k = 0; k < kB2QWords; k++) {
                x[k] = 0u;
                if (w0 + k < p.W) {
                    x[k] = __ldcg(f + w0 + k);
                    f[w0 + k] = 0u;
                    other[w0 + k] = 0u;
                }
            }
        }
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < kB2QWords; k++) cnt += __popc(x[k]);
        const int incl = warp_inclusive_scan(cnt);
        if (lane == 31) s_wtot[wib] = incl;
        __syncthreads();
        if (threadIdx.x < 32) {
            const int c = lane < nwb ? s_wtot[lane] : 0;
            const int wi = warp_inclusive_scan(c);
            const int total = __shfl_sync(kFull, wi, 31);
            unsigned long long b = 0;
            if (lane == 0 && total) b = atomicAdd(tail, (unsigned long long)total);
            if (lane < nwb) s_wtot[lane] = wi - c;
            if (lane == 0) s_qb = b;
        }
        __syncthreads();
        long long pos = (long long)s_qb + s_wtot[wib] + incl - cnt;
#pragma unroll
        for (int k = 0; k < kB2QWords; k++) {
            unsigned y = x[k];
            while (y) {
                const int bit = __ffs(y) - 1;
                y &= y - 1;
                q[pos++] = (int)((w0 + k) * 32 + bit);
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ bottom-up

// ids[t] for a run-time t (0 <= t < N) as a chain of selects: indexing the
// array at run time would move the whole window to the stack every round
template <int N>
__device__ __forceinline__ int pick(const int (&ids)[N], int t) {
    int v = ids[0];
#pragma unroll
    for (int i = 1; i < N; i++)
        if (t == i) v = ids[i];
    return v;
}

__device__ __forceinline__ bool in_frontier(const unsigned* f, int v) {
    return (__ldcg(f + (v >> 5)) >> (v & 31)) & 1u;
}

// Append a warp's staged long-list entries with one atomicAdd.
__device__ __forceinline__ void long_flush(WarpStage& st, int* longlist, unsigned long long* longcnt) {
    if (st.cnt == 0) return;
    __syncwarp();
    unsigned long long base = 0;
    if (lane_id() == 0) base = atomicAdd(longcnt, (unsigned long long)st.cnt);
    base = __shfl_sync(kFull, base, 0);
    for (int i = lane_id(); i < st.cnt; i += 32) longlist[base + i] = st.buf[i];
    __syncwarp();
    st.cnt = 0;
}

// Bottom-up, phase A.  A warp takes 32 completed-bitmap words (1024
// vertices) at a time and compacts the unvisited ones with a warp prefix sum;
// each lane then handles one searcher per round: its row offsets, one aligned
// window of 8 ids (two int4 loads) and 8 frontier probes.  The rounds are
// software-pipelined three deep -- while round r's probes run, round r+1's
// window and round r+2's offsets are already in flight -- so each round costs
// about one L2 probe latency instead of two DRAM round trips.  A searcher
// whose row continues past the window without a hit goes on the long list
// (phase B).  Found vertices are collected per word in shared memory and
// written as whole next-frontier / completed words (the warp owns its words).
__device__ __forceinline__ int bu_locate(int k, int T, int incl, int excl, unsigned todo, long long ch) {
    int j = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1) {
        const int c = __shfl_sync(kFull, incl, j + step - 1);
        if (c <= k) j += step;
    }
    const int exj = __shfl_sync(kFull, excl, j);
    const unsigned tj = __shfl_sync(kFull, todo, j);
    if (k >= T) return -1;
    return (int)((ch * 32 + j) * 32 + (long long)__fns(tj, 0, k - exj + 1));
}

__device__ void bu_phase_a(const SingleParams& p, int d, const unsigned* fcur, unsigned* fnext, int* longlist,
                           unsigned long long* longcnt, unsigned long long& acc_n, unsigned long long& acc_m,
                           unsigned long long& acc_sc, unsigned long long& acc_ex) {
    __shared__ unsigned s_next[kBlock / 32][32];
    const int lane = lane_id(), wib = threadIdx.x >> 5;
    const long long nchunk = (p.W + 31) / 32;
    const int4 z4 = make_int4(0, 0, 0, 0);
    s_next[wib][lane] = 0u;
    WarpStage lst = warp_stage();   // long-list entries, appended in batches
    __syncwarp();
    const long long gw = gtid() >> 5, nw = gthreads() >> 5;
    for (long long ch = gw; ch < nchunk; ch += nw) {
        const long long w = ch * 32 + lane;
        const unsigned cw = (w < p.W) ? __ldcg(p.visited + w) : kFull;
        const unsigned todo = ~cw;
        const int cnt = __popc(todo);
        const int incl = warp_inclusive_scan(cnt);
        const int T = __shfl_sync(kFull, incl, 31);
        const int excl = incl - cnt;
        // pipeline prologue: round 0 offsets + window, round 1 offsets
        int u0 = bu_locate(lane, T, incl, excl, todo, ch);
        long long s0 = 0, e0 = 0;
        if (u0 >= 0) {
            bu_row_of_stream(p, u0, s0, e0);
        }
        int4 xa0 = z4, xb0 = z4;
        if (u0 >= 0 && e0 > s0) {
            const int4* src = reinterpret_cast<const int4*>(p.cols_bu + (s0 & ~3LL));
            xa0 = ld_stream4(src);
            if (kWin == 8 && (s0 & ~3LL) + 4 < e0) xb0 = ld_stream4(src + 1);
        }
        int u1 = bu_locate(32 + lane, T, incl, excl, todo, ch);
        long long s1 = 0, e1 = 0;
        if (u1 >= 0) {
            bu_row_of_stream(p, u1, s1, e1);
        }
        for (int base = 0; base < T; base += 32) {
            // round r+2: offsets
            const int u2 = bu_locate(base + 64 + lane, T, incl, excl, todo, ch);
            long long s2 = 0, e2 = 0;
            if (u2 >= 0) {
                bu_row_of_stream(p, u2, s2, e2);
            }
            // round r+1: window
            int4 xa1 = z4, xb1 = z4;
            if (u1 >= 0 && e1 > s1) {
                const int4* src = reinterpret_cast<const int4*>(p.cols_bu + (s1 & ~3LL));
                xa1 = ld_stream4(src);
                if (kWin == 8 && (s1 & ~3LL) + 4 < e1) xb1 = ld_stream4(src + 1);
            }
            // round r: probes
            bool to_long = false;
            if (u0 >= 0) {
                const long long rb = s0 & ~3LL;
                const int ids[8] = {xa0.x, xa0.y, xa0.z, xa0.w, xb0.x, xb0.y, xb0.z, xb0.w};
                // probe the first id alone (on most levels it is the hit), the rest of
                // the window only on a miss: L2 requests, not latency, bound this loop
                const int t0 = (int)(s0 - rb);
                const int first_id = (t0 == 0) ? xa0.x : (t0 == 1) ? xa0.y : (t0 == 2) ? xa0.z : xa0.w;
                unsigned hb = 0;
                if (e0 > s0 && in_frontier(fcur, first_id)) {
                    hb = 1u << t0;
                } else {
#pragma unroll
                    for (int t = 0; t < kWin; t++) {
                        const long long q = rb + t;
                        if (t > t0 && q < e0 && in_frontier(fcur, ids[t])) hb |= 1u << t;
                    }
                }
                acc_sc += 1;
                if (hb) {
                    const int t = __ffs(hb) - 1;
                    acc_ex += (unsigned long long)(rb + t - s0 + 1);
                    acc_m += (unsigned long long)(e0 - s0);
                    if (p.parent) p.parent[u0] = pick(ids, t);
                    set_level(p, u0, d + 1);
                    atomicOr(&s_next[wib][(u0 >> 5) - ch * 32], 1u << (u0 & 31));
                } else if (rb + kWin < e0) {
                    to_long = true;       // examinations counted by phase B
                } else {
                    acc_ex += (unsigned long long)(e0 - s0);
                }
            }
            const unsigned lm = __ballot_sync(kFull, to_long);
            if (lm) {
                if (to_long) lst.buf[lst.cnt + __popc(lm & lanemask_lt())] = u0;
                lst.cnt += __popc(lm);
                if (lst.cnt > kStage - 32) long_flush(lst, longlist, longcnt);
            }
            u0 = u1;
            s0 = s1;
            e0 = e1;
            xa0 = xa1;
            xb0 = xb1;
            u1 = u2;
            s1 = s2;
            e1 = e2;
        }
        __syncwarp();
        const unsigned nx = s_next[wib][lane];
        if (w < p.W) {
            fnext[w] = nx;
            if (nx) p.visited[w] = cw | nx;
        }
        acc_n += (unsigned long long)__popc(nx);
        s_next[wib][lane] = 0u;
        __syncwarp();
    }
    long_flush(lst, longlist, longcnt);
}

// Bottom-up over the hub-first rows, phase A: the first probe of every
// searcher.  Algorithm 2 scans a searcher's row in order and stops at the first
// neighbour in the frontier; over the hub-first rows that first neighbour is
// the hit for most searchers on R-MAT graphs.  So phase A reads, per searcher,
// only first[v] (the first id of its row, bit 31: more neighbours follow), a
// per-vertex plane.  A warp takes 32 completed-bitmap words (1024 vertices) at a
// time and compacts their searchers onto lanes (a warp prefix sum), one
// searcher per lane per round, software-pipelined three deep: round r+2's plane
// value and round r+1's frontier probe are in flight while round r consumes its
// probe.  Hits are collected per word in shared memory and written as whole
// next-frontier words (the warp owns its chunk's words).  A hit stores no
// parent: its parent is first[v], recorded by one bit of pfirst (the final pass
// writes the parent array).  A miss with more neighbours goes on the miss list
// (phase B); a degree-1 miss is done.
//
// No degree is read for a hit: the degree sum of the new frontier is m_u minus
// the degree sum of the searchers left unvisited, which phases A-C count
// (acc_left), and a searcher left unvisited has had its whole row examined.
constexpr int kHead = 7;          // ids in a row head
constexpr unsigned kMore = 0x80000000u;

__device__ __forceinline__ unsigned frontier_word(const unsigned* f, int v) { return __ldcg(f + (v >> 5)); }

constexpr int kMissPerLane = 2;   // misses whose row heads a lane reads together
#ifndef BFS_INLINE_MISSES
#define BFS_INLINE_MISSES 128
#endif
// A chunk with at most this many first-probe misses resolves them in its own
// warp at the end of the chunk (two steps of kMissPerLane per lane at most: no miss-list
// round trip, no global atomics, and the random head reads overlap other warps'
// first probes); a chunk with more sends them to the miss list, which phase B
// spreads over every warp.
constexpr int kInlineMisses = BFS_INLINE_MISSES;

// The first-probe misses of a warp's current chunk (staged in st.buf[0..cnt)):
// each lane takes kMissPerLane of them per step and reads their 32-byte row
// heads together (degree and the first seven ids), then probes ids 1..6 in row
// order.  A hit goes into `cmiss`, the chunk's words of such hits in shared
// memory (merged into the chunk's next-frontier words when they are written,
// so no global atomics, and kept out of `pfirst`: these parents are stored); a
// row that goes on is appended to the long list (phase C resumes it at 7).
__device__ __forceinline__ void chunk_misses(const SingleParams& p, int d, const unsigned* fcur, WarpStage& st,
                                             unsigned* cmiss, long long ch, int* longlist, unsigned long long* longcnt,
                                             unsigned long long& acc_left, unsigned long long& acc_ex) {
    const int lane = lane_id();
    __syncwarp();
    for (int i0 = 0; i0 < st.cnt; i0 += 32 * kMissPerLane) {
        int u[kMissPerLane];
        int4 a[kMissPerLane], b[kMissPerLane];
#pragma unroll
        for (int r = 0; r < kMissPerLane; r++) {
            const int i = i0 + r * 32 + lane;
            u[r] = i < st.cnt ? st.buf[i] : -1;
            a[r] = b[r] = make_int4(0, 0, 0, 0);
            if (u[r] >= 0) ld_stream8(p.heads + 8 * (long long)u[r], a[r], b[r]);
        }
#pragma unroll
        for (int r = 0; r < kMissPerLane; r++) {
            bool to_long = false;
            if (u[r] >= 0) {
                const int deg = a[r].x;
                const int ids[kHead] = {a[r].y, a[r].z, a[r].w, b[r].x, b[r].y, b[r].z, b[r].w};
                unsigned hit = 0;
#pragma unroll
                for (int t = 1; t < kHead; t++)
                    if (t < deg && in_frontier(fcur, ids[t])) hit |= 1u << t;
                if (hit) {
                    const int t = __ffs(hit) - 1;
                    const int v = u[r];
                    acc_ex += (unsigned long long)(t + 1);
                    if (p.parent) p.parent[v] = pick(ids, t);
                    set_level(p, v, d + 1);
                    atomicOr(cmiss + ((v >> 5) - ch * 32), 1u << (v & 31));
                } else if (deg > kHead) {
                    to_long = true;       // examinations counted by phase C
                } else {
                    acc_ex += (unsigned long long)deg;
                    acc_left += (unsigned long long)deg;
                }
            }
            const unsigned lm = __ballot_sync(kFull, to_long);
            if (lm) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(longcnt, (unsigned long long)__popc(lm));
                base = __shfl_sync(kFull, base, 0);
                if (to_long) longlist[base + __popc(lm & lanemask_lt())] = u[r];
            }
        }
    }
    __syncwarp();
    st.cnt = 0;
}

__device__ void bu_compact(const SingleParams& p, int d, const unsigned* fcur, unsigned* fnext, int* misslist,
                           unsigned long long* misscnt, unsigned long long* misscnt_inline, int* longlist,
                           unsigned long long* longcnt,
                           unsigned long long& acc_n, unsigned long long& acc_left, unsigned long long& acc_sc,
                           unsigned long long& acc_ex) {
    __shared__ unsigned s_cnext[kBlock / 32][32];
    __shared__ unsigned s_cmiss[kBlock / 32][32];   // the chunk's hits among misses it resolved itself
    s_cmiss[threadIdx.x >> 5][lane_id()] = 0u;
    const int lane = lane_id(), wib = threadIdx.x >> 5;
    unsigned short* list = g_list[wib];
    const long long nchunk = (p.W + 31) / 32;
    s_cnext[wib][lane] = 0u;
    WarpStage mst = warp_stage();
    unsigned long long nmiss_w = 0;   // warp-uniform
    __syncwarp();
    const long long gw = gtid() >> 5, nw = gthreads() >> 5;
    for (long long ch = gw; ch < nchunk; ch += nw) {
        const long long w = ch * 32 + lane;
        const unsigned cw = (w < p.W) ? __ldcg(p.visited + w) : kFull;
        unsigned todo = ~cw;
        const int cnt = __popc(todo);
        const int incl = warp_inclusive_scan(cnt);
        const int T = __shfl_sync(kFull, incl, 31);
        int pos = incl - cnt;
        while (todo) {
            const int b = __ffs(todo) - 1;
            todo &= todo - 1;
            list[pos++] = (unsigned short)(lane * 32 + b);
        }
        __syncwarp();
        const long long vbase = ch * 1024;
        // round r's searcher: vertex vbase + list[32 r + lane], or none past T
        auto who = [&](int r) -> int { const int k = 32 * r + lane; return k < T ? (int)(vbase + list[k]) : -1; };
        auto plane = [&](int u) -> int { return u >= 0 ? ld_stream32(p.first + u) : 0; };
        // software pipeline: plane values three rounds ahead, frontier probes one round ahead
        int f0 = plane(who(0)), f1 = plane(who(1)), f2 = plane(who(2));
        unsigned pw0 = who(0) >= 0 ? frontier_word(fcur, f0 & (int)~kMore) : 0u;
        const int R = (T + 31) / 32;
        for (int r = 0; r < R; r++) {
            const int f3 = plane(who(r + 3));
            const unsigned pw1 = who(r + 1) >= 0 ? frontier_word(fcur, f1 & (int)~kMore) : 0u;
            const int u0 = who(r);
            const bool act = u0 >= 0;
            const bool hit = act && ((pw0 >> (f0 & 31)) & 1u);
            const bool miss = act && !hit && ((unsigned)f0 & kMore);
            if (act) {
                acc_sc += 1;
                acc_ex += (unsigned long long)(hit || !miss);
                if (hit) {
                    set_level(p, u0, d + 1);
                    if (!p.pfirst && p.parent) p.parent[u0] = f0 & (int)~kMore;
                    atomicOr(&s_cnext[wib][(u0 >> 5) - ch * 32], 1u << (u0 & 31));
                } else if (!miss) {
                    acc_left += 1;
                }
            }
            const unsigned mm = __ballot_sync(kFull, miss);
            if (mm) {
                if (miss) mst.buf[mst.cnt + __popc(mm & lanemask_lt())] = u0;
                mst.cnt += __popc(mm);
                if (mst.cnt > kStage - 32) long_flush(mst, misslist, misscnt);
            }
            f0 = f1;
            f1 = f2;
            f2 = f3;
            pw0 = pw1;
        }
        if (mst.cnt > kInlineMisses) {
            long_flush(mst, misslist, misscnt);
        } else if (mst.cnt > 0) {
            nmiss_w += (unsigned long long)mst.cnt;
            chunk_misses(p, d, fcur, mst, s_cmiss[wib], ch, longlist, longcnt, acc_left, acc_ex);
        }
        __syncwarp();
        const unsigned nf = s_cnext[wib][lane];   // first-probe hits: parent = the plane entry
        const unsigned nx = nf | s_cmiss[wib][lane];
        s_cmiss[wib][lane] = 0u;
        if (w < p.W) {
            fnext[w] = nx;
            if (nx) {
                p.visited[w] = cw | nx;
                if (p.pfirst && nf) atomicOr(p.pfirst + w, nf);
            }
        }
        acc_n += (unsigned long long)__popc(nx);
        s_cnext[wib][lane] = 0u;
        __syncwarp();
    }
    // misses resolved here, for the level's record
    if (lane == 0 && nmiss_w) atomicAdd(misscnt_inline, nmiss_w);
}

// Bottom-up over the hub-first rows, phase B: the miss list.  Each lane takes
// kMissPerLane searchers per step and reads their 32-byte row heads (degree and
// the first seven ids, one 256-bit load each, all in flight together), then
// probes ids 1..6 in row order.  A hit writes its parent directly; the next-
// frontier and completed words are shared with other warps here, hence
// atomicOr.  A searcher with more than seven neighbours and no hit among them
// goes on the long list (phase C resumes its row at position 7).
__device__ void bu_misses(const SingleParams& p, int d, const unsigned* fcur, unsigned* fnext, const int* misslist,
                          long long nmiss, int* longlist, unsigned long long* longcnt, unsigned long long& acc_n,
                          unsigned long long& acc_left, unsigned long long& acc_ex) {
    const int lane = lane_id();
    WarpStage lst = warp_stage();
    const long long gw = gtid() >> 5, nw = gthreads() >> 5;
    constexpr int kStep = 32 * kMissPerLane;
    for (long long base = gw * kStep; base < nmiss; base += nw * kStep) {
        int u[kMissPerLane];
        int4 a[kMissPerLane], b[kMissPerLane];
#pragma unroll
        for (int r = 0; r < kMissPerLane; r++) {
            const long long i = base + r * 32 + lane;
            u[r] = -1;
            a[r] = b[r] = make_int4(0, 0, 0, 0);
            if (i < nmiss) {
                u[r] = __ldcg(misslist + i);
                ld_stream8(p.heads + 8 * (long long)u[r], a[r], b[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < kMissPerLane; r++) {
            bool to_long = false;
            if (u[r] >= 0) {
                const int deg = a[r].x;
                const int ids[kHead] = {a[r].y, a[r].z, a[r].w, b[r].x, b[r].y, b[r].z, b[r].w};
                unsigned hit = 0;
#pragma unroll
                for (int t = 1; t < kHead; t++)
                    if (t < deg && in_frontier(fcur, ids[t])) hit |= 1u << t;
                if (hit) {
                    const int t = __ffs(hit) - 1;
                    const int v = u[r];
                    acc_ex += (unsigned long long)(t + 1);
                    acc_n += 1;
                    if (p.parent) p.parent[v] = pick(ids, t);
                    set_level(p, v, d + 1);
                    atomicOr(fnext + (v >> 5), 1u << (v & 31));
                    atomicOr(p.visited + (v >> 5), 1u << (v & 31));
                } else if (deg > kHead) {
                    to_long = true;       // examinations counted by phase C
                } else {
                    acc_ex += (unsigned long long)deg;
                    acc_left += (unsigned long long)deg;
                }
            }
            const unsigned lm = __ballot_sync(kFull, to_long);
            if (lm) {
                if (to_long) lst.buf[lst.cnt + __popc(lm & lanemask_lt())] = u[r];
                lst.cnt += __popc(lm);
                if (lst.cnt > kStage - 32) long_flush(lst, longlist, longcnt);
            }
        }
    }
    long_flush(lst, longlist, longcnt);
}

// Bottom-up, phase B: the long list.  Groups of 4 lanes take one searcher
// each (8 per warp); a group reads 16 ids per step (one int4 per lane, in row
// order) and stops at the first frontier neighbour: the lowest lane of the
// group with a hit, its lowest id -- so parents stay the minimum-id ones.
// Next-frontier and completed words are shared across warps here, hence
// atomicOr.
// With count_left, acc_m receives the degrees of the searchers left unvisited
// (the hub-first sweep's accounting); otherwise those of the ones found.
__device__ void bu_phase_b(const SingleParams& p, int d, const unsigned* fcur, unsigned* fnext, const int* longlist,
                           long long nlong, int skip, bool count_left, unsigned long long& acc_n,
                           unsigned long long& acc_m, unsigned long long& acc_ex) {
    const int lane = lane_id(), grp = lane >> 2, gl = lane & 3;
    const long long gw = gtid() >> 5, nw = gthreads() >> 5;
    for (long long base = gw * 8; base < nlong; base += nw * 8) {
        const long long i = base + grp;
        int u = -1;
        long long s0 = 0, e0 = 0, pos = 0;
        if (i < nlong) {
            u = __ldcg(longlist + i);
            bu_row_of(p, u, s0, e0);
            pos = ((s0 + skip) & ~3LL) + 4 * gl;
        }
        long long hitpos = -1;
        int pv = -1;
        bool live = u >= 0;
        while (__any_sync(kFull, live)) {
            unsigned hb = 0;
            int4 x = make_int4(0, 0, 0, 0);
            if (live && pos < e0) {
                x = ld_stream4(reinterpret_cast<const int4*>(p.cols_bu + pos));
                const int ids[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int t = 0; t < 4; t++)
                    if (pos + t < e0 && in_frontier(fcur, ids[t])) hb |= 1u << t;
            }
            const unsigned any = __ballot_sync(kFull, hb != 0);
            const unsigned gm = (any >> (grp * 4)) & 0xFu;
            const long long gstart = pos - 4 * gl;   // group's position this step
            // every lane runs both shuffles (full-mask warp primitives must be convergent):
            // each lane offers its own first hit, the group reads its lowest lane with one
            const int t_own = hb ? __ffs(hb) - 1 : 0;
            const int v_own = (t_own == 0) ? x.x : (t_own == 1) ? x.y : (t_own == 2) ? x.z : x.w;
            const int first = gm ? __ffs(gm) - 1 : 0;
            const int t_src = __shfl_sync(kFull, t_own, grp * 4 + first);
            const int v_src = __shfl_sync(kFull, v_own, grp * 4 + first);
            if (live) {
                if (gm) {
                    hitpos = gstart + 4 * first + t_src;
                    pv = v_src;
                    live = false;
                } else if (gstart + 16 >= e0) {
                    live = false;
                }
            }
            pos += 16;
        }
        if (u >= 0 && gl == 0) {
            if (hitpos >= 0) {
                acc_ex += (unsigned long long)(hitpos - s0 + 1);
                if (!count_left) acc_m += (unsigned long long)(e0 - s0);
                acc_n += 1;
                if (p.parent) p.parent[u] = pv;
                set_level(p, u, d + 1);
                atomicOr(fnext + (u >> 5), 1u << (u & 31));
                atomicOr(p.visited + (u >> 5), 1u << (u & 31));
            } else {
                acc_ex += (unsigned long long)(e0 - s0);
                if (count_left) acc_m += (unsigned long long)(e0 - s0);
            }
        }
    }
}

// ------------------------------------------------------------------ cluster levels
//
// A top-down level with a small frontier costs the grid a chain of dependent
// global round trips (queue, offsets, columns, claim, queue tail) and a grid
// barrier of several hundred CTAs: on a graph of large diameter (a mesh or a
// torus) that fixed cost is the whole search.  While the frontier stays small,
// the CTAs of thread-block cluster 0 run the levels alone: the frontier lives
// in their shared memory, each CTA takes an equal share of it from whichever
// CTA discovered it (distributed shared memory), a frontier entry carries its
// row's offset and degree (read once, when the vertex is claimed), and a
// level ends at the hardware cluster barrier.  The other CTAs wait on a flag
// until the frontier outgrows the cluster (or the direction rule picks
// bottom-up), when the cluster writes the frontier back to the global queue
// and the grid takes over at that level.  Levels, parents, claims and the
// per-level counters are those of the grid's top-down step.

constexpr int kCluMaxC = 16;
constexpr int kCluBig = 128;            // largest degree of a vertex in a cluster level's frontier
constexpr int kCluEdgesPerCta = 4096;   // a cluster level takes at most this many edges per CTA
constexpr long long kCluAutoMaxDeg = 32;   // automatic: cluster levels on graphs of max degree <= this
constexpr int kCluDegShift = 40;         // a frontier entry's row: offset | degree << 40
struct CluEntry {
    unsigned long long row;   // first column index of the row | min(degree, 2^24 - 1) << 40
    int v;                    // vertex
    int par;                  // its parent (-1: not known), whose edge the expansion skips
};
static_assert(sizeof(CluEntry) == 16, "a frontier entry is one 16-byte load");
__device__ __forceinline__ unsigned long long clu_row(long long s, long long deg) {
    return (unsigned long long)s | ((unsigned long long)min(deg, (long long)0xFFFFFF) << kCluDegShift);
}
constexpr int kCluCap = (int)(sizeof(g_list) / 2 / sizeof(CluEntry));   // entries per CTA buffer (half of g_list)
constexpr unsigned long long kCluCntMask = 0x7FFFull;   // entry count field of a summary word
static_assert(kCluCap <= 0x7FFF, "entry count field");

__device__ __forceinline__ unsigned clu_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned clu_id() {
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned clu_nranks() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// every thread of every CTA of the cluster, from warp-uniform code; orders
// shared-memory (local and remote) writes before it against reads after it.
// The aligned form (the warp executes it together, as after the __syncwarp)
// keeps the kernel's register allocation intact; the unaligned form does not.
__device__ __forceinline__ void clu_sync() {
    __syncwarp();
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// the shared::cluster address of `local` in CTA `rank` of this cluster
__device__ __forceinline__ unsigned clu_map(const void* local, unsigned rank) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(local);
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void clu_ld_entry(unsigned addr, long long& s, int& deg, int& v, int& par) {
    unsigned long long a, b;
    asm volatile("ld.shared::cluster.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "r"(addr) : "memory");
    s = (long long)(a & ((1ull << kCluDegShift) - 1ull));
    deg = (int)(a >> kCluDegShift);
    v = (int)(unsigned)b;
    par = (int)(unsigned)(b >> 32);
}
__device__ __forceinline__ void clu_st64(unsigned addr, unsigned long long x) {
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(x) : "memory");
}

// Per-CTA summaries of a frontier, pushed by each CTA into every CTA of the
// cluster: [parity][rank] = {entries | heavy << 15 | spilled << 32, degree sum}.
__shared__ unsigned long long g_csum[2][kCluMaxC][2];

struct CluState {
    int d;                 // next level for the grid (done: the last level)
    long long nf, mf, mu, reached;
    bool done;
};

// Expand level L of the cluster's frontier (entries in `cur` of every CTA,
// counts in g_csum[b]) into this CTA's `next` buffer.  Entries past the
// buffer spill to the front of queue0 (the level after is then the grid's).
__device__ void clu_expand(const SingleParams& p, int L, int C, int r, int b, long long nf, const CluEntry* cur,
                           CluEntry* next, int* s_lcnt, unsigned long long& acc_m, unsigned& acc_h) {
    const int lane = lane_id(), nwb = blockDim.x >> 5, wib = threadIdx.x >> 5;
    const long long cw = (long long)r * nwb + wib, ncw = (long long)C * nwb;
    const long long per = nf >= ncw * 32 ? 32 : max(1LL, (nf + ncw - 1) / ncw);
    for (long long base = cw * per; base < nf; base += ncw * per) {
        const long long i = base + lane;
        int u = 0, deg = 0, pu = -1;
        long long s = 0;
        if (lane < per && i < nf) {
            // owner CTA of entry i (the entries are numbered CTA by CTA)
            int q = 0;
            long long acc = 0;
            while (q < C - 1) {
                const long long c = (long long)(g_csum[b][q][0] & kCluCntMask);
                if (i < acc + c) break;
                acc += c;
                q++;
            }
            if (i - acc < kCluCap) clu_ld_entry(clu_map(cur + (i - acc), (unsigned)q), s, deg, u, pu);
        }
        const int incl = warp_inclusive_scan(deg);
        const int total = __shfl_sync(kFull, incl, 31);
        const int excl = incl - deg;
        // four edges per lane per round: the column reads, then the claims, then
        // the claimed rows' offsets, each four in flight together; the edge back
        // to a vertex's parent is known visited and skipped
        for (int k0 = 0; k0 < total; k0 += 128) {
            int v[4], uu[4];
            bool act[4];
#pragma unroll
            for (int q4 = 0; q4 < 4; q4++) {
                const int k = k0 + q4 * 32 + lane;
                int j = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const int c = __shfl_sync(kFull, incl, j + step - 1);
                    if (c <= k) j += step;
                }
                const long long sj = __shfl_sync(kFull, s, j);
                const int exj = __shfl_sync(kFull, excl, j);
                const int pj = __shfl_sync(kFull, pu, j);
                uu[q4] = __shfl_sync(kFull, u, j);
                act[q4] = k < total;
                v[q4] = act[q4] ? __ldg(p.cols + sj + (k - exj)) : 0;
                act[q4] = act[q4] && v[q4] != pj;
            }
            bool cl[4];
#pragma unroll
            for (int q4 = 0; q4 < 4; q4++) {
                const unsigned bit = 1u << (v[q4] & 31);
                cl[q4] = act[q4] && !(atomicOr(p.visited + (v[q4] >> 5), bit) & bit);
            }
            long long rs[4], re[4];
#pragma unroll
            for (int q4 = 0; q4 < 4; q4++) {
                rs[q4] = 0;
                re[q4] = 0;
                if (cl[q4]) row_of(p, v[q4], rs[q4], re[q4]);
            }
            const int mine = (int)cl[0] + (int)cl[1] + (int)cl[2] + (int)cl[3];
            const int inc2 = warp_inclusive_scan(mine);
            const int tot2 = __shfl_sync(kFull, inc2, 31);
            if (tot2 == 0) continue;
            int pos = 0;
            if (lane == 0) pos = atomicAdd(s_lcnt, tot2);
            pos = __shfl_sync(kFull, pos, 0) + inc2 - mine;
#pragma unroll
            for (int q4 = 0; q4 < 4; q4++) {
                if (!cl[q4]) continue;
                const int vv = v[q4];
                if (p.parent) p.parent[vv] = uu[q4];
                set_level(p, vv, L + 1);
                const long long dg = re[q4] - rs[q4];
                acc_m += (unsigned long long)dg;
                acc_h |= dg > (long long)p.clu_big;
                if (dg > 0) asm volatile("prefetch.global.L2 [%0];" ::"l"(p.cols + rs[q4]));
                if (pos < kCluCap) {
                    CluEntry e;
                    e.row = clu_row(rs[q4], dg);
                    e.v = vv;
                    e.par = uu[q4];
                    next[pos] = e;
                } else {
                    const unsigned long long sp = atomicAdd(&p.ctrl->clu_spill, 1ull);
                    p.queue0[sp] = vv;
                }
                pos++;
            }
        }
    }
}

// Levels d0, d0+1, ... run by the CTAs of cluster 0 (every thread of them
// calls).  Enters with the frontier of level d0 in `qcur` (nf0 vertices, mf0
// edges, none above the degree cap); leaves when the search is done or the
// grid must take the next level, with the state for it in `out` and, for the
// waiting CTAs, in the control block.
__device__ void cluster_levels(const SingleParams& p, const int* qcur, int d0, long long nf0, long long mf0,
                               long long mu0, long long reached0, unsigned long long epi, uint64_t t_start,
                               CluState& out) {
    __shared__ int s_lcnt, s_lh;
    __shared__ unsigned long long s_lm;
    Ctrl* c = p.ctrl;
    const int C = p.clu_c, r = (int)clu_rank(), tid = threadIdx.x, nth = blockDim.x;
    const int lane = lane_id(), wib = tid >> 5;
    const bool lead = blockIdx.x == 0 && tid == 0;
    CluEntry* const buf0 = reinterpret_cast<CluEntry*>(&g_list[0][0]);
    CluEntry* const buf1 = buf0 + kCluCap;
    // this CTA's share of the entry frontier, with the rows' offsets and degrees
    {
        const long long lo = nf0 * r / C, hi = nf0 * (r + 1) / C;
        for (long long i = lo + tid; i < hi; i += nth) {
            const int u = __ldcg(qcur + i);
            long long rs, re;
            row_of(p, u, rs, re);
            CluEntry e;
            e.row = clu_row(rs, re - rs);
            e.v = u;
            e.par = -1;
            buf0[i - lo] = e;
        }
        if (tid < C) {
            const long long cnt = nf0 * (tid + 1) / C - nf0 * tid / C;
            g_csum[0][tid][0] = (unsigned long long)cnt;
            g_csum[0][tid][1] = tid == 0 ? (unsigned long long)mf0 : 0ull;
        }
        if (tid == 0) {
            s_lcnt = 0;
            s_lh = 0;
            s_lm = 0;
        }
    }
    clu_sync();
    int L = d0, b = 0;
    long long mu = mu0, reached = reached0, pnf = 0, pmf = 0;
    while (true) {
        long long nf = 0, mf = 0, spill = 0;
        bool heavy = false;
        for (int q = 0; q < C; q++) {
            const unsigned long long w0 = g_csum[b][q][0];
            nf += (long long)(w0 & kCluCntMask) + (long long)(w0 >> 32);
            spill += (long long)(w0 >> 32);
            heavy |= ((w0 >> 15) & 1ull) != 0;
            mf += (long long)g_csum[b][q][1];
        }
        if (L > d0) {
            if (lead && L - 1 < p.rec_cap) {
                bfs_level_record rec;
                rec.dir = TD;
                rec.misses = 0;
                rec.nf = pnf;
                rec.mf = pmf;
                rec.nnext = nf;
                rec.mnext = mf;
                rec.scanned = 0;
                rec.examined = pmf;
                rec.t_ns = (long long)(globaltimer_ns() - t_start);
                rec.aux = -1;   // a cluster level
                rec.t_mid_ns = 0;
                p.rec[L - 1] = rec;
            }
            if (nf > 0) {
                reached += nf;
                mu -= mf;
            }
        }
        const bool done = nf == 0;
        const bool leave = done || spill > 0 || heavy || nf > p.clu_nf || mf > p.clu_mf ||
                           decide_dir(p, TD, nf, mf, mu, L) != TD;
        if (leave) {
            if (!done) {
                // the frontier back to queue0: spilled entries first, then CTA by CTA
                long long pre = spill;
                for (int q = 0; q < r; q++) pre += (long long)(g_csum[b][q][0] & kCluCntMask);
                const int mine = (int)(g_csum[b][r][0] & kCluCntMask);
                const CluEntry* cur = b ? buf1 : buf0;
                for (int i = tid; i < mine; i += nth) p.queue0[pre + i] = cur[i].v;
            }
            out.d = done ? L - 1 : L;
            out.nf = nf;
            out.mf = mf;
            out.mu = mu;
            out.reached = reached;
            out.done = done;
            if (lead) {
                // the grid resumes at level L with every per-level counter slot clear
                for (int k = 0; k < 3; k++) {
                    c->tail[k] = 0;
                    c->accn[k] = 0;
                    c->accm[k] = 0;
                    c->scanned[k] = 0;
                    c->examined[k] = 0;
                    c->ntask[k] = 0;
                    c->nmiss[k] = 0;
                    c->nmiss_in[k] = 0;
                    c->dsum_out[k] = 0;
                    c->dsum_in[k] = 0;
                    c->heavy[k] = 0;
                }
                c->clu_spill = 0;
                c->clu_d = out.d;
                c->clu_nf = nf;
                c->clu_mf = mf;
                c->clu_mu = mu;
                c->clu_reached = reached;
                c->clu_done = done ? 1 : 0;
            }
            // every CTA's queue, level, parent and claim writes, then the hand-over
            __threadfence();
            clu_sync();
            if (lead) asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(&c->clu_gen), "l"(epi) : "memory");
            return;
        }
        if (lead) asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(&c->clu_prog), "l"((unsigned long long)L)
                               : "memory");
        unsigned long long am = 0;
        unsigned ah = 0;
        clu_expand(p, L, C, r, b, nf, b ? buf1 : buf0, b ? buf0 : buf1, &s_lcnt, am, ah);
        am = warp_sum(am);
        const bool hw = __any_sync(kFull, ah != 0);
        if (lane == 0) {
            if (am) atomicAdd(&s_lm, am);
            if (hw) s_lh = 1;
        }
        __syncthreads();
        if (wib == 0) {
            const int lc = s_lcnt;
            const unsigned long long lm = s_lm;
            const int lh = s_lh;
            const int cnt = lc < kCluCap ? lc : kCluCap;
            const unsigned long long w0 = (unsigned long long)cnt | ((unsigned long long)(lh ? 1 : 0) << 15) |
                                          ((unsigned long long)(lc - cnt) << 32);
            if (lane < C) {
                clu_st64(clu_map(&g_csum[b ^ 1][r][0], (unsigned)lane), w0);
                clu_st64(clu_map(&g_csum[b ^ 1][r][1], (unsigned)lane), lm);
            }
            __syncwarp();
            if (lane == 0) {
                s_lcnt = 0;
                s_lh = 0;
                s_lm = 0;
            }
        }
        clu_sync();
        pnf = nf;
        pmf = mf;
        L++;
        b ^= 1;
    }
}

// A CTA outside cluster 0 during cluster levels: thread 0 waits for episode
// `epi` to end (giving up only when the cluster makes no progress for the
// run's time limit); then every thread reads the state the cluster left.
__device__ bool clu_wait(const SingleParams& p, unsigned long long epi, CluState& out) {
    __shared__ int s_ok;
    Ctrl* c = p.ctrl;
    if (threadIdx.x == 0) {
        uint64_t t0 = globaltimer_ns();
        unsigned long long last = ~0ull;
        int ok = 1;
        unsigned spins = 0;
        while (true) {
            if (ld_acquire64(&c->clu_gen) >= epi) break;
            if (ld_relaxed64(&c->b.count) & kAbortBit) {
                ok = 0;
                break;
            }
            const unsigned long long pr = ld_relaxed64(&c->clu_prog);
            const uint64_t now = globaltimer_ns();
            if (pr != last) {
                last = pr;
                t0 = now;
            } else if (now - t0 > p.timeout_ns) {
                raise_status(&c->b, kDevTimeout);
                ok = 0;
                break;
            }
            __nanosleep(++spins < 16 ? 128 : 512);
        }
        s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return false;
    out.d = (int)ld_relaxed64(reinterpret_cast<const unsigned long long*>(&c->clu_d));
    out.nf = (long long)ld_relaxed64(reinterpret_cast<const unsigned long long*>(&c->clu_nf));
    out.mf = (long long)ld_relaxed64(reinterpret_cast<const unsigned long long*>(&c->clu_mf));
    out.mu = (long long)ld_relaxed64(reinterpret_cast<const unsigned long long*>(&c->clu_mu));
    out.reached = (long long)ld_relaxed64(reinterpret_cast<const unsigned long long*>(&c->clu_reached));
    out.done = ld_relaxed64(reinterpret_cast<const unsigned long long*>(&c->clu_done)) != 0;
    return true;
}

// ------------------------------------------------------------------ kernel

__global__ void __launch_bounds__(kBlock, BFS_MIN_BLOCKS) bfs_single_kernel(SingleParams p) {
    Ctrl* c = p.ctrl;
    if (blockIdx.x == 0 && threadIdx.x == 0) c->t_enter = globaltimer_ns();
    init_phase(p);
    if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) c->t_init = globaltimer_ns();
    if (p.nroots == 1 && gtid() == 0) {
        if (p.parent) p.parent[p.root0] = p.root0;
        set_level(p, p.root0, 0);
    }
    if (p.nroots > 1) {
        seed_roots_phase(p);
        if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
    }
    long long nf = p.nroots;
    long long mf = (long long)ld_relaxed64(&c->accm[0]);
    long long mu = p.nnz - mf;
    if (p.directed) {
        // m_u sums in-degrees: the edges a bottom-up step could still examine
        long long rin = 0;
        if (p.nroots == 1) {
            long long s0, e0;
            bu_row_of(p, p.root0, s0, e0);
            rin = e0 - s0;
        } else {
            rin = (long long)ld_relaxed64(&c->dsum_in[0]);
        }
        mu = p.nnz - rin;
    }
    long long reached = nf;
    int prev = TD, qsel = 0, bsel = 0, d = 0;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const uint64_t t_start = lead ? globaltimer_ns() : 0;
    // cluster levels only in a launch whose clusters have the size the parameters name
    const bool clu_on = p.clu_c > 1 && clu_nranks() == (unsigned)p.clu_c;
    unsigned long long epi = 0;
    int no_clu = -1;   // the level a cluster episode just handed back (the grid takes it)
    while (true) {
        const int dir = decide_dir(p, prev, nf, mf, mu, d);
        if (clu_on && dir == TD && prev == TD && d != no_clu && nf <= p.clu_nf && mf <= p.clu_mf &&
            (d == 0 ? mf <= (long long)p.clu_big : ld_relaxed64(&c->heavy[d % 3]) == 0ull)) {
            epi++;
            CluState cs;
            if (clu_id() == 0) {
                cluster_levels(p, qsel ? p.queue1 : p.queue0, d, nf, mf, mu, reached, epi, t_start, cs);
            } else if (!clu_wait(p, epi, cs)) {
                return;
            }
            d = cs.d;
            reached = cs.reached;
            if (cs.done) break;
            nf = cs.nf;
            mf = cs.mf;
            mu = cs.mu;
            prev = TD;
            qsel = 0;   // the frontier is back in queue0
            no_clu = d;
            continue;
        }
        const int scur = d % 3, snext = (d + 1) % 3, sfree = (d + 2) % 3;
        if (lead) {
            c->tail[sfree] = 0;
            c->accn[sfree] = 0;
            c->accm[sfree] = 0;
            c->scanned[sfree] = 0;
            c->examined[sfree] = 0;
            c->ntask[sfree] = 0;
            c->nmiss[sfree] = 0;
            c->nmiss_in[sfree] = 0;
            c->dsum_out[sfree] = 0;
            c->dsum_in[sfree] = 0;
            c->heavy[sfree] = 0;
        }
        long long nf_next, scanned = 0, examined = mf, aux = 0, misses = 0;
        uint64_t t_mid = 0;
        int* qcur = qsel ? p.queue1 : p.queue0;
        int* qnext = qsel ? p.queue0 : p.queue1;
        unsigned* fcur = bsel ? p.front1 : p.front0;
        unsigned* fnext = bsel ? p.front0 : p.front1;
        if (dir == TD) {
            if (prev == BU) {
                bitmap_to_queue(p, fcur, fnext, qcur, &c->tail[scur]);
                if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            }
            unsigned long long am = 0, ah = 0;
            unsigned long long* gh = clu_on ? &c->heavy[snext] : nullptr;
            // a directed graph sums the new frontier's degrees after the level
            const bool nodeg = p.directed != 0;
            td_phase(p, d, qcur, nf, qnext, snext, nodeg, am, ah);
            block_add4(ah, am, 0, 0, gh, &c->accm[snext], nullptr, nullptr);
            if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            const long long nt = (long long)ld_relaxed64(&c->ntask[snext]);
            aux = nt;
            if (lead) t_mid = globaltimer_ns();
            if (nt > 0) {
                unsigned long long am2 = 0, ah2 = 0;
                task_phase(p, d, nt, qnext, snext, nodeg, am2, ah2);
                block_add4(ah2, am2, 0, 0, gh, &c->accm[snext], nullptr, nullptr);
                if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            }
            nf_next = (long long)ld_relaxed64(&c->tail[snext]);
            qsel ^= 1;
        } else {
            if (prev == TD) {
                queue_to_bitmap(p, qcur, nf, fcur);
                if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            }
            // over the hub-first rows accm[snext] collects the degrees of the searchers
            // left unvisited (the new frontier's degree sum is m_u minus that), over the
            // id-ordered rows those of the vertices found
            unsigned long long an = 0, am = 0, asc = 0, aex = 0;
            // the queues are idle during bottom-up levels (a preceding queue -> bitmap
            // conversion ended at the barrier above)
            int* longlist = qnext;
            int* misslist = qcur;
            if (p.first)
                bu_compact(p, d, fcur, fnext, misslist, &c->nmiss[snext], &c->nmiss_in[snext], longlist,
                           &c->ntask[snext], an, am, asc, aex);
            else
                bu_phase_a(p, d, fcur, fnext, longlist, &c->ntask[snext], an, am, asc, aex);
            block_add4(an, am, asc, aex, &c->accn[snext], &c->accm[snext], &c->scanned[snext],
                       &c->examined[snext]);
            if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            if (lead) t_mid = globaltimer_ns();
            if (p.first) {
                const long long nmiss = (long long)ld_relaxed64(&c->nmiss[snext]);
                misses = nmiss + (long long)ld_relaxed64(&c->nmiss_in[snext]);
                if (nmiss > 0) {
                    unsigned long long bn = 0, bm = 0, bex = 0;
                    bu_misses(p, d, fcur, fnext, misslist, nmiss, longlist, &c->ntask[snext], bn, bm, bex);
                    block_add4(bn, bm, 0, bex, &c->accn[snext], &c->accm[snext], nullptr, &c->examined[snext]);
                    if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
                }
            }
            const long long nlong = (long long)ld_relaxed64(&c->ntask[snext]);
            aux = nlong;
            if (nlong > 0) {
                unsigned long long bn = 0, bm = 0, bex = 0;
                bu_phase_b(p, d, fcur, fnext, longlist, nlong, p.first ? kHead : kWin, p.first != nullptr, bn, bm,
                           bex);
                block_add4(bn, bm, 0, bex, &c->accn[snext], &c->accm[snext], nullptr, &c->examined[snext]);
                if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            }
            nf_next = (long long)ld_relaxed64(&c->accn[snext]);
            scanned = (long long)ld_relaxed64(&c->scanned[snext]);
            examined = (long long)ld_relaxed64(&c->examined[snext]);
            bsel ^= 1;
        }
        const long long macc = (long long)ld_relaxed64(&c->accm[snext]);
        long long mf_next = (dir == BU && p.first) ? mu - macc : macc;
        long long mu_drop = mf_next;   // undirected: in- and out-degree sums coincide
        if (p.directed) {
            unsigned long long so = 0, si = 0;
            if (dir == TD)
                frontier_degree_sums(p, qsel ? p.queue1 : p.queue0, nf_next, nullptr, so, si);
            else
                frontier_degree_sums(p, nullptr, 0, bsel ? p.front1 : p.front0, so, si);
            block_add4(so, si, 0, 0, &c->dsum_out[snext], &c->dsum_in[snext], nullptr, nullptr);
            if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            mf_next = (long long)ld_relaxed64(&c->dsum_out[snext]);
            mu_drop = (long long)ld_relaxed64(&c->dsum_in[snext]);
        }
        if (lead && d < p.rec_cap) {
            bfs_level_record r;
            r.dir = dir;
            r.misses = (int)misses;
            r.nf = nf;
            r.mf = mf;
            r.nnext = nf_next;
            r.mnext = mf_next;
            r.scanned = scanned;
            r.examined = examined;
            r.t_ns = (long long)(globaltimer_ns() - t_start);
            r.aux = aux;
            r.t_mid_ns = t_mid ? (long long)(t_mid - t_start) : 0;
            p.rec[d] = r;
        }
        if (nf_next == 0) break;
        reached += nf_next;
        mu -= mu_drop;
        nf = nf_next;
        mf = mf_next;
        prev = dir;
        d++;
    }
    if (lead) {
        c->num_levels = d + 1;
        c->reached = reached;
        c->t_levels = globaltimer_ns();
    }
    // every level ended at a grid barrier, so all staged bytes are visible here
    if (p.parent_mode == BFS_PARENT_MIN_ID && p.parent && p.level) {
        min_parent_pass(p);
        if (p.lv8 && !grid_sync(&c->b, p.expected, p.timeout_ns)) return;
    }
    if (p.lv8) {
        materialise(p);
        // the last CTA through the final pass stamps its end
        __syncthreads();
        if (threadIdx.x == 0 && atomicAdd(&c->done_ctas, 1ull) == (unsigned long long)gridDim.x - 1ull)
            c->t_done = globaltimer_ns();
    }
}

// ------------------------------------------------------------------ DCSC tiles

// Words of vertex block b that exist (the last block may run past n).
__device__ __forceinline__ long long block_words(const SingleParams& p, int b) {
    const long long w0 = (long long)b * p.Bw;
    const long long w1 = min(w0 + p.Bw, p.W);
    return w1 > w0 ? w1 - w0 : 0;
}

// Top-down on tiles (b, *) (Algorithm 3's local discovery, t = A_bj * f_j):
// every CTA reads the whole frontier queue, finds each frontier vertex k's
// column in its tile (b, block(k)) by binary search over JC, and claims the
// column's rows -- all in block b, so claims are CTA-local bit operations on
// the block's visited words held in shared memory (the sparse accumulator).
__device__ void td_dcsc_phase(const SingleParams& p, int d, const int* qcur, long long nf, int* qnext, int snext,
                              unsigned* s_own, unsigned long long& acc_m) {
    const int b = blockIdx.x, lane = lane_id();
    const long long nbw = block_words(p, b), wbase = (long long)b * p.Bw;
    for (long long w = threadIdx.x; w < nbw; w += blockDim.x) s_own[w] = __ldcg(p.visited + wbase + w);
    __syncthreads();
    unsigned long long* tail = &p.ctrl->tail[snext];
    WarpStage st = warp_stage_dcsc();
    const int wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
    for (long long base = (long long)wib * 32; base < nf; base += (long long)nwb * 32) {
        const long long i = base + lane;
        int k = -1;
        long long cs = 0, ce = 0;
        if (i < nf) {
            k = __ldcg(qcur + i);
            const long long j = k / p.B;
            const long long t = (long long)b * p.nb + j;
            long long lo = __ldg(p.tile_ptr + t), hi = __ldg(p.tile_ptr + t + 1);
            const int kl = (int)(k - j * p.B);
            while (lo < hi) {
                const long long mid = (lo + hi) >> 1;
                if (__ldg(p.jc + mid) < kl) lo = mid + 1; else hi = mid;
            }
            if (lo < __ldg(p.tile_ptr + t + 1) && __ldg(p.jc + lo) == kl) {
                cs = __ldg(p.cp + lo);
                ce = __ldg(p.cp + lo + 1);
            }
        }
        const int mydeg = (int)(ce - cs);
        const int incl = warp_inclusive_scan(mydeg);
        const int total = __shfl_sync(kFull, incl, 31);
        const int excl = incl - mydeg;
        for (int k0 = 0; k0 < total; k0 += 32) {
            const int kk = k0 + lane;
            int j = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int c = __shfl_sync(kFull, incl, j + step - 1);
                if (c <= kk) j += step;
            }
            const long long cj = __shfl_sync(kFull, cs, j);
            const int exj = __shfl_sync(kFull, excl, j);
            const int kj = __shfl_sync(kFull, k, j);
            bool claimed = false;
            int u = 0;
            if (kk < total) {
                const int ul = __ldg(p.ir + cj + (kk - exj));
                const unsigned bit = 1u << (ul & 31);
                if (!(s_own[ul >> 5] & bit)) claimed = !(atomicOr(s_own + (ul >> 5), bit) & bit);
                u = (int)((long long)b * p.B + ul);
            }
            const unsigned cm = __ballot_sync(kFull, claimed);
            if (cm) {
                if (claimed) {
                    st.buf[st.cnt + __popc(cm & lanemask_lt())] = u;
                    if (p.parent) p.parent[u] = kj;
                    if (p.level) p.level[u] = d + 1;
                }
                st.cnt += __popc(cm);
                if (st.cnt > kStage - 32) stage_flush(p, st, qnext, tail, acc_m);
            }
        }
    }
    stage_flush(p, st, qnext, tail, acc_m);
    __syncthreads();
    for (long long w = threadIdx.x; w < nbw; w += blockDim.x) p.visited[wbase + w] = s_own[w];
}

// Bottom-up on tiles (*, b) (Algorithm 4's sub-steps without messages): the
// CTA owning block b walks the p tiles of its column of the grid; each
// searcher u of block b (a column of the tile: the matrix is symmetric) not
// yet completed scans its rows in block i and stops at the first one in the
// frontier.  The completed bits of block b live in shared memory for the whole
// level.  With minimum-id parents the tiles run 0..p-1 with the frontier
// segment of block i staged in shared memory and a CTA barrier between tiles
// (so a searcher stops at its first frontier neighbour in id order); with any
// parent the tile order rotates with b, the segment is probed in L2, and tiles
// follow one another without barriers.
__device__ void bu_dcsc_phase(const SingleParams& p, int d, const unsigned* fcur, unsigned* fnext, unsigned* s_own,
                              unsigned* s_seg, unsigned long long& acc_n, unsigned long long& acc_m,
                              unsigned long long& acc_sc, unsigned long long& acc_ex) {
    const int b = blockIdx.x;
    const long long nbw = block_words(p, b), wbase = (long long)b * p.Bw;
    for (long long w = threadIdx.x; w < nbw; w += blockDim.x) {
        const unsigned x = __ldcg(p.visited + wbase + w);
        s_own[w] = x;
        acc_sc += (unsigned long long)__popc(~x);
    }
    if (p.parent_mode != BFS_PARENT_MIN_ID) {
        // any parent will do: tiles in rotated order with no staging and no barrier
        // between them (the frontier segment is probed in L2), four column entries per
        // thread in flight.  A searcher found in two tiles at once gets either parent.
        for (int t = 0; t < p.nb; t++) {
            const int i = (b + t) % p.nb;
            const unsigned* fseg = fcur + (long long)i * p.Bw;
            const long long tt = (long long)i * p.nb + b;
            const long long lo = __ldg(p.tile_ptr + tt), hi = __ldg(p.tile_ptr + tt + 1);
            for (long long x0 = lo + threadIdx.x; x0 < hi; x0 += 4LL * blockDim.x) {
                int ul[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const long long x = x0 + (long long)k * blockDim.x;
                    ul[k] = x < hi ? __ldg(p.jc + x) : -1;
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    if (ul[k] < 0 || ((s_own[ul[k] >> 5] >> (ul[k] & 31)) & 1u)) continue;
                    const long long x = x0 + (long long)k * blockDim.x;
                    const long long e0 = __ldg(p.cp + x), e1 = __ldg(p.cp + x + 1);
                    for (long long e = e0; e < e1; e++) {
                        const int vl = __ldg(p.ir + e);
                        if ((__ldcg(fseg + (vl >> 5)) >> (vl & 31)) & 1u) {
                            const long long u = (long long)b * p.B + ul[k];
                            if (p.parent) p.parent[u] = (int)((long long)i * p.B + vl);
                            if (p.level) p.level[u] = d + 1;
                            atomicOr(s_own + (ul[k] >> 5), 1u << (ul[k] & 31));
                            acc_ex += (unsigned long long)(e - e0 + 1);
                            break;
                        }
                        if (e + 1 == e1) acc_ex += (unsigned long long)(e1 - e0);
                    }
                }
            }
        }
    }
    for (int t = 0; t < p.nb && p.parent_mode == BFS_PARENT_MIN_ID; t++) {
        const int i = t;
        const long long ibw = block_words(p, i), ibase = (long long)i * p.Bw;
        __syncthreads();
        for (long long w = threadIdx.x; w < ibw; w += blockDim.x) s_seg[w] = __ldcg(fcur + ibase + w);
        __syncthreads();
        const long long tt = (long long)i * p.nb + b;
        const long long lo = __ldg(p.tile_ptr + tt), hi = __ldg(p.tile_ptr + tt + 1);
        for (long long x = lo + threadIdx.x; x < hi; x += blockDim.x) {
            const int ul = __ldg(p.jc + x);
            if ((s_own[ul >> 5] >> (ul & 31)) & 1u) continue;
            const long long e0 = __ldg(p.cp + x), e1 = __ldg(p.cp + x + 1);
            for (long long e = e0; e < e1; e++) {
                const int vl = __ldg(p.ir + e);
                if ((s_seg[vl >> 5] >> (vl & 31)) & 1u) {
                    const long long u = (long long)b * p.B + ul;
                    if (p.parent) p.parent[u] = (int)((long long)i * p.B + vl);
                    if (p.level) p.level[u] = d + 1;
                    atomicOr(s_own + (ul >> 5), 1u << (ul & 31));
                    acc_ex += (unsigned long long)(e - e0 + 1);
                    break;
                }
                if (e + 1 == e1) acc_ex += (unsigned long long)(e1 - e0);
            }
        }
    }
    __syncthreads();
    for (long long w = threadIdx.x; w < nbw; w += blockDim.x) {
        const unsigned old = __ldcg(p.visited + wbase + w);
        const unsigned now = s_own[w];
        const unsigned nw = now & ~old;
        fnext[wbase + w] = nw;
        if (nw) p.visited[wbase + w] = now;
        acc_n += (unsigned long long)__popc(nw);
        unsigned bits = nw;
        while (bits) {
            const int bt = __ffs(bits) - 1;
            bits &= bits - 1;
            const long long u = (wbase + w) * 32 + bt;
            acc_m += (unsigned long long)deg_of(p, u);
        }
    }
}

__global__ void __launch_bounds__(kDBlock, 1) bfs_dcsc_kernel(SingleParams p) {
    extern __shared__ unsigned dyn[];
    unsigned* s_own = dyn;
    unsigned* s_seg = dyn + p.Bw;
    Ctrl* c = p.ctrl;
    init_phase(p);
    if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
    if (p.nroots == 1 && gtid() == 0) {
        if (p.parent) p.parent[p.root0] = p.root0;
        if (p.level) p.level[p.root0] = 0;
    }
    if (p.nroots > 1) {
        seed_roots_phase(p);
        if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
    }
    long long nf = p.nroots;
    long long mf = (long long)ld_relaxed64(&c->accm[0]);
    long long mu = p.nnz - mf;
    long long reached = nf;
    int prev = TD, qsel = 0, bsel = 0, d = 0;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const uint64_t t_start = lead ? globaltimer_ns() : 0;
    while (true) {
        const int dir = decide_dir(p, prev, nf, mf, mu, d);
        const int scur = d % 3, snext = (d + 1) % 3, sfree = (d + 2) % 3;
        if (lead) {
            c->tail[sfree] = 0;
            c->accn[sfree] = 0;
            c->accm[sfree] = 0;
            c->scanned[sfree] = 0;
            c->examined[sfree] = 0;
            c->ntask[sfree] = 0;
        }
        long long nf_next, scanned = 0, examined = mf;
        int* qcur = qsel ? p.queue1 : p.queue0;
        int* qnext = qsel ? p.queue0 : p.queue1;
        unsigned* fcur = bsel ? p.front1 : p.front0;
        unsigned* fnext = bsel ? p.front0 : p.front1;
        if (dir == TD) {
            if (prev == BU) {
                bitmap_to_queue(p, fcur, fnext, qcur, &c->tail[scur]);
                if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            }
            unsigned long long am = 0;
            td_dcsc_phase(p, d, qcur, nf, qnext, snext, s_own, am);
            block_add4(0, am, 0, 0, nullptr, &c->accm[snext], nullptr, nullptr);
            if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            nf_next = (long long)ld_relaxed64(&c->tail[snext]);
            qsel ^= 1;
        } else {
            if (prev == TD) {
                queue_to_bitmap(p, qcur, nf, fcur);
                if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            }
            unsigned long long an = 0, am = 0, asc = 0, aex = 0;
            bu_dcsc_phase(p, d, fcur, fnext, s_own, s_seg, an, am, asc, aex);
            block_add4(an, am, asc, aex, &c->accn[snext], &c->accm[snext], &c->scanned[snext], &c->examined[snext]);
            if (!grid_sync(&c->b, p.expected, p.timeout_ns)) return;
            nf_next = (long long)ld_relaxed64(&c->accn[snext]);
            scanned = (long long)ld_relaxed64(&c->scanned[snext]);
            examined = (long long)ld_relaxed64(&c->examined[snext]);
            bsel ^= 1;
        }
        const long long mf_next = (long long)ld_relaxed64(&c->accm[snext]);
        if (lead && d < p.rec_cap) {
            bfs_level_record r;
            r.dir = dir;
            r.misses = 0;
            r.nf = nf;
            r.mf = mf;
            r.nnext = nf_next;
            r.mnext = mf_next;
            r.scanned = scanned;
            r.examined = examined;
            r.t_ns = (long long)(globaltimer_ns() - t_start);
            r.aux = 0;
            r.t_mid_ns = 0;
            p.rec[d] = r;
        }
        if (nf_next == 0) break;
        reached += nf_next;
        mu -= mf_next;
        nf = nf_next;
        mf = mf_next;
        prev = dir;
        d++;
    }
    if (lead) {
        c->num_levels = d + 1;
        c->reached = reached;
    }
    if (p.parent_mode == BFS_PARENT_MIN_ID && p.parent && p.level) min_parent_pass(p);
}

// ------------------------------------------------------------------ allocation-free variant

// Work buffers of bfs_run_csr_noalloc live in this file-scope device array, so
// that entry point never allocates.  Limits: n <= kStaticMaxN, nnz <=
// kStaticMaxNnz.  Every call shares it (calls that overlap on the GPU race);
// each call re-initialises everything it reads.
constexpr long long kStaticMaxN = 1LL << 20;
constexpr long long kStaticMaxNnz = 1LL << 24;
constexpr long long kStaticW = kStaticMaxN / 32;
constexpr long long kStaticTasks = kStaticMaxNnz / kChunk + kStaticMaxNnz / 64 + 1024;   // default chunk
constexpr int kStaticRec = 64;
constexpr size_t kStaticCtrlOff = 0;
constexpr size_t kStaticIsoOff = (sizeof(Ctrl) + 255) / 256 * 256;   // control block slot
constexpr size_t kStaticVisOff = kStaticIsoOff + 4 * kStaticW;
constexpr size_t kStaticF0Off = kStaticVisOff + 4 * kStaticW;
constexpr size_t kStaticF1Off = kStaticF0Off + 4 * kStaticW;
constexpr size_t kStaticQ0Off = kStaticF1Off + 4 * kStaticW;
constexpr size_t kStaticQ1Off = kStaticQ0Off + 4 * (kStaticMaxN + 64);
constexpr size_t kStaticTaskOff = kStaticQ1Off + 4 * (kStaticMaxN + 64);
constexpr size_t kStaticRecOff = kStaticTaskOff + sizeof(Task) * kStaticTasks;
constexpr size_t kStaticBytes = kStaticRecOff + sizeof(bfs_level_record) * kStaticRec;
static_assert(kStaticQ1Off % 16 == 0 && kStaticTaskOff % 16 == 0 && kStaticRecOff % 8 == 0, "alignment");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kStaticBytes];

// bit v set when deg(v) = 0 or v >= n (vertices that never search)
__global__ void k_static_isolated(const long long* __restrict__ off, long long n, long long W, unsigned* iso) {
    const long long nth = (long long)gridDim.x * blockDim.x;
    for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < W; w += nth) {
        unsigned x = 0;
        for (int b = 0; b < 32; b++) {
            const long long v = w * 32 + b;
            if (v >= n || off[v + 1] == off[v]) x |= 1u << b;
        }
        iso[w] = x;
    }
}

}  // namespace bfsk

// ====================================================================== host

namespace bfsrt {

using bfsk::Ctrl;
using bfsk::SingleParams;
using bfsk::Task;

bfs_status single_prepare(bfs_graph* g, cudaStream_t s) { return single_prepare_work(g, g->single, s, 0); }

// Work buffers of one single-source search state on graph g; grid > 0 caps the
// launch grid (a server runs several searches side by side with small grids).
bfs_status single_prepare_work(bfs_graph* g, SingleWork& w, cudaStream_t s, int grid) {
    if (w.ready) return BFS_OK;
    const long long n = g->n, W = g->W;
    // chunks of >= kMinChunk edges of vertices of degree > 64: at most nnz/64 + nnz/64 tasks
    const long long task_cap = g->nnz / bfsk::kMinChunk + g->nnz / 64 + 1024;
    const int rec_cap = 1 << 16;
    struct Item { void** p; size_t bytes; };
    Item items[] = {
        {(void**)&w.visited, sizeof(unsigned) * (size_t)W},
        {(void**)&w.front0, sizeof(unsigned) * (size_t)W},
        {(void**)&w.front1, sizeof(unsigned) * (size_t)W},
        {(void**)&w.queue0, sizeof(int) * (size_t)(n + 32)},
        {(void**)&w.queue1, sizeof(int) * (size_t)(n + 32)},
        {(void**)&w.lv8, (size_t)W * 32},   // one byte per vertex, rounded up to whole bitmap words
        {(void**)&w.pfirst, sizeof(unsigned) * (size_t)W},
        {(void**)&w.tasks, sizeof(Task) * (size_t)task_cap},
        {(void**)&w.ctrl, sizeof(Ctrl)},
        {(void**)&w.records, sizeof(bfs_level_record) * (size_t)rec_cap},
    };
    size_t total = 0;
    for (auto& it : items) {
        *it.p = mem_of(g, w).alloc(it.bytes, s);
        if (!*it.p) {
            for (auto& jt : items)
                if (*jt.p) { mem_of(g, w).release(*jt.p, jt.bytes, s); *jt.p = nullptr; }
            return fail(BFS_ERR_OOM, "single-source work buffers: device allocation failed");
        }
        total += it.bytes;
    }
    w.task_cap = task_cap;
    w.rec_cap = rec_cap;
    w.bytes = total;
    int nb = 0;
    BFS_CUDA_TRY(cudaFuncSetAttribute(bfsk::bfs_single_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)bfsk::kSingleDynSmem));
    BFS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bfsk::bfs_single_kernel, bfsk::kBlock,
                                                               bfsk::kSingleDynSmem));
    if (nb < 1) return fail(BFS_ERR_UNSUPPORTED, "BFS kernel cannot be resident on this device");
    w.block = bfsk::kBlock;
    w.grid = nb * g->sm_count;
    if (grid > 0 && grid < w.grid) w.grid = grid;
    BFS_CUDA_TRY(cudaMemsetAsync(w.ctrl, 0, sizeof(Ctrl), s));
    w.ready = true;
    return BFS_OK;
}

void single_release(bfs_graph* g) { single_release_work(g, g->single); }

void single_release_work(bfs_graph* g, SingleWork& w) {
    if (!w.ready) return;
    const long long n = g->n, W = g->W;
    mem_of(g, w).release(w.visited, sizeof(unsigned) * (size_t)W, nullptr);
    mem_of(g, w).release(w.front0, sizeof(unsigned) * (size_t)W, nullptr);
    mem_of(g, w).release(w.front1, sizeof(unsigned) * (size_t)W, nullptr);
    mem_of(g, w).release(w.queue0, sizeof(int) * (size_t)(n + 32), nullptr);
    mem_of(g, w).release(w.queue1, sizeof(int) * (size_t)(n + 32), nullptr);
    mem_of(g, w).release(w.lv8, (size_t)W * 32, nullptr);
    mem_of(g, w).release(w.pfirst, sizeof(unsigned) * (size_t)W, nullptr);
    if (w.level_scratch) mem_of(g, w).release(w.level_scratch, sizeof(int) * (size_t)n, nullptr);
    mem_of(g, w).release(w.tasks, sizeof(Task) * (size_t)w.task_cap, nullptr);
    mem_of(g, w).release(w.ctrl, sizeof(Ctrl), nullptr);
    mem_of(g, w).release(w.records, sizeof(bfs_level_record) * (size_t)w.rec_cap, nullptr);
    DeviceAlloc* keep = w.mem;   // the allocator choice outlives the buffers
    w = SingleWork();
    w.mem = keep;
}

bfs_status single_launch(bfs_graph* g, const int32_t* roots_host, int32_t k, int32_t* parent,
                         int32_t* level, const bfs_options& opt, cudaStream_t s) {
    return single_launch_work(g, g->single, roots_host, k, parent, level, opt, s);
}

bfs_status single_launch_work(bfs_graph* g, SingleWork& w, const int32_t* roots_host, int32_t k, int32_t* parent,
                              int32_t* level, const bfs_options& opt, cudaStream_t s) {
    if (opt.parent_mode == BFS_PARENT_MIN_ID && parent && !level) {
        // minimum-id parents are picked by level; keep them in a private array
        if (!w.level_scratch) {
            w.level_scratch = (int*)mem_of(g, w).alloc(sizeof(int) * (size_t)g->n, s);
            if (!w.level_scratch) return fail(BFS_ERR_OOM, "MIN_ID parents: level scratch allocation failed");
        }
        level = w.level_scratch;
    }
    SingleParams p;
    p.off = reinterpret_cast<const long long*>(g->offsets);
    p.cols = g->cols;
    const bool hub = opt.bu_rows == BFS_BU_ROWS_HUB_FIRST && g->cols_hf;
    p.cols_bu = g->directed ? g->cols_in : (hub ? g->cols_hf : g->cols);
    p.off_bu = reinterpret_cast<const long long*>(g->directed ? g->offsets_in : g->offsets);
    p.deg8_in = g->deg8_in;
    p.directed = g->directed ? 1 : 0;
    p.heads = (hub && g->bu_heads && g->bu_first) ? g->bu_heads : nullptr;
    p.first = p.heads ? g->bu_first : nullptr;
    p.deg8 = g->deg8;
    p.isolated = g->isolated;
    p.n = g->n;
    p.nnz = g->nnz;
    p.W = g->W;
    p.parent = parent;
    p.level = level;
    // staged outputs and the final whole-sector pass (CSR kernel, some output requested)
    p.lv8 = (opt.layout == BFS_LAYOUT_DCSC_TILED || (!parent && !level)) ? nullptr : w.lv8;
    p.pfirst = (p.lv8 && p.first) ? w.pfirst : nullptr;   // only a plane sweep sets its bits
    p.visited = w.visited;
    p.front0 = w.front0;
    p.front1 = w.front1;
    p.queue0 = w.queue0;
    p.queue1 = w.queue1;
    p.tasks = reinterpret_cast<Task*>(w.tasks);
    p.task_cap = w.task_cap;
    p.ctrl = reinterpret_cast<Ctrl*>(w.ctrl);
    p.rec = w.records;
    p.rec_cap = w.rec_cap;
    p.root0 = roots_host[0];
    p.nroots = k;
    p.mode = opt.mode;
    p.alpha = opt.alpha;
    p.beta = opt.beta;
    p.parent_mode = opt.parent_mode;
    p.big_deg = opt.td_big_degree > 0 ? opt.td_big_degree : 96;
    p.td_chunk = opt.td_chunk > 0 ? opt.td_chunk : bfsk::kDefaultChunk;
    p.clu_c = 1;
    p.clu_big = 0;
    p.clu_nf = 0;
    p.clu_mf = 0;
    p.seed = opt.seed;
    p.timeout_ns = (unsigned long long)(opt.timeout_ms > 0 ? opt.timeout_ms : 10000) * 1000000ull;
    const unsigned extra = (unsigned)(g->debug_barrier_extra > 0 ? g->debug_barrier_extra : 0);
    p.expected = (unsigned)w.grid + extra;
    p.tile_ptr = nullptr;
    p.jc = nullptr;
    p.cp = nullptr;
    p.ir = nullptr;
    p.nb = 0;
    p.B = 0;
    p.Bw = 0;
    const bool dcsc = opt.layout == BFS_LAYOUT_DCSC_TILED;
    int grid = w.grid, block = w.block;
    if (opt.ctas_per_sm > 0 && (long long)opt.ctas_per_sm * g->sm_count < grid) {
        grid = opt.ctas_per_sm * g->sm_count;
        p.expected = (unsigned)grid + extra;
    }
    size_t dyn = bfsk::kSingleDynSmem;
    if (dcsc) {
        const DcscTiles& D = g->dcsc;
        p.tile_ptr = reinterpret_cast<const long long*>(D.tile_ptr);
        p.jc = D.jc;
        p.cp = reinterpret_cast<const long long*>(D.cp);
        p.ir = D.ir;
        p.nb = D.num_blocks;
        p.B = D.block_size;
        p.Bw = D.block_size / 32;
        dyn = sizeof(unsigned) * 2 * (size_t)p.Bw;
        BFS_CUDA_TRY(cudaFuncSetAttribute(bfsk::bfs_dcsc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        int occ = 0;
        BFS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bfsk::bfs_dcsc_kernel, bfsk::kDBlock, dyn));
        if (occ < 1 || (long long)occ * g->sm_count < D.num_blocks)
            return fail(BFS_ERR_UNSUPPORTED, "DCSC kernel: the tile grid cannot be co-resident on this device");
        grid = D.num_blocks;
        block = bfsk::kDBlock;
        p.expected = (unsigned)grid + extra;
    }
    // cluster levels (CSR, undirected): the launch in clusters of C CTAs, as many as fit
    int C = 1;
    if (!dcsc && !g->directed)
        C = opt.cluster_size > 0 ? opt.cluster_size : (g->max_degree <= bfsk::kCluAutoMaxDeg ? 16 : 1);
    while (C > 1 && C > grid) C >>= 1;   // a small grid (a server's executor) is one cluster at most
    if (C > 1) {
        int li = 0;
        while ((1 << li) < C) li++;
        if (w.clu_grid[li] == 0) {
            BFS_CUDA_TRY(cudaFuncSetAttribute(bfsk::bfs_single_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = (unsigned)C;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3((unsigned)C);
            cfg.blockDim = dim3((unsigned)block);
            cfg.dynamicSmemBytes = dyn;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int ncl = 0;
            BFS_CUDA_TRY(cudaOccupancyMaxActiveClusters(&ncl, bfsk::bfs_single_kernel, &cfg));
            w.clu_grid[li] = ncl > 0 ? ncl * C : -1;
        }
        const int g2 = (grid < w.clu_grid[li] ? grid : w.clu_grid[li]) / C * C;
        if (g2 < C) {
            C = 1;   // clusters of this size cannot be resident, or the grid is smaller: plain launch
        } else {
            grid = g2;
            p.expected = (unsigned)grid + extra;
        }
    }
    if (C > 1) {
        p.clu_c = C;
        p.clu_big = bfsk::kCluBig;
        p.clu_nf = (long long)C * (bfsk::kCluCap / 2);
        p.clu_mf = (long long)C * bfsk::kCluEdgesPerCta;
    }
    BFS_CUDA_TRY(cudaMemsetAsync(w.ctrl, 0, sizeof(Ctrl), s));
    if (k > 1) BFS_CUDA_TRY(cudaMemcpyAsync(w.queue0, roots_host, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, s));
    if (C > 1) {
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        at[1].id = cudaLaunchAttributeCooperative;
        at[1].val.cooperative = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3((unsigned)block);
        cfg.dynamicSmemBytes = dyn;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 2;
        BFS_CUDA_TRY(cudaLaunchKernelEx(&cfg, bfsk::bfs_single_kernel, p));
        return BFS_OK;
    }
    void* args[] = {&p};
    const void* fn = dcsc ? (const void*)bfsk::bfs_dcsc_kernel : (const void*)bfsk::bfs_single_kernel;
    BFS_CUDA_TRY(cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, dyn, s));
    return BFS_OK;
}

size_t single_ctrl_bytes() { return sizeof(Ctrl); }
unsigned single_ctrl_status(const void* ctrl_host) { return reinterpret_cast<const Ctrl*>(ctrl_host)->b.status; }

bfs_status single_collect(bfs_graph* g, cudaStream_t s, bfs_stats* stats) {
    SingleWork& w = g->single;
    Ctrl c;
    BFS_CUDA_TRY(cudaMemcpyAsync(&c, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    BFS_CUDA_TRY(cudaStreamSynchronize(s));
    if (c.b.status == bfsk::kDevTimeout)
        return fail(BFS_ERR_TIMEOUT, "device grid barrier wait ran out of time; outputs are undefined");
    if (c.b.status == bfsk::kDevOverflow)
        return fail(BFS_ERR_CUDA, "top-down chunk task list overflowed (internal sizing error)");
    if (stats) {
        stats->num_levels = (int32_t)c.num_levels;
        stats->t_init_ns = c.t_init > c.t_enter ? (int64_t)(c.t_init - c.t_enter) : 0;
        stats->t_final_ns = c.t_done > c.t_levels ? (int64_t)(c.t_done - c.t_levels) : 0;
        stats->vertices_reached = c.reached;
        const int nrec = (int)std::min<long long>(c.num_levels, (long long)w.rec_cap);
        const int ncopy = std::min(nrec, stats->levels_capacity);
        stats->edges_examined = 0;
        if (nrec > 0) {
            bfs_level_record* tmp = new (std::nothrow) bfs_level_record[nrec];
            if (!tmp) return fail(BFS_ERR_OOM, "host allocation for level records");
            cudaError_t e = cudaMemcpy(tmp, w.records, sizeof(bfs_level_record) * (size_t)nrec, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) { delete[] tmp; return cuda_fail(e, "cudaMemcpy(level records)"); }
            for (int i = 0; i < nrec; i++) stats->edges_examined += tmp[i].examined;
            if (stats->levels && ncopy > 0) memcpy(stats->levels, tmp, sizeof(bfs_level_record) * (size_t)ncopy);
            delete[] tmp;
        }
    }
    return BFS_OK;
}

}  // namespace bfsrt

// ====================================================================== allocation-free entry point

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};   // device address of g_noalloc_scratch, per device
int g_noalloc_grid[64] = {};
int g_noalloc_sms[64] = {};
}  // namespace

extern "C" bfs_status bfs_run_csr_noalloc(const int64_t* row_offsets, const int32_t* col_ids, int64_t n, int64_t nnz,
                                          int32_t root, int32_t* parent_dev, int32_t* level_dev, void* stream) {
    using namespace bfsrt;
    if (!row_offsets || (nnz > 0 && !col_ids)) return fail(BFS_ERR_INVALID, "row_offsets / col_ids must not be NULL");
    if (n < 1 || n > bfsk::kStaticMaxN)
        return fail(BFS_ERR_INVALID, "bfs_run_csr_noalloc: n must lie in [1, " + std::to_string(bfsk::kStaticMaxN) +
                                         "] (its scratch is a fixed device array)");
    if (nnz < 0 || nnz > bfsk::kStaticMaxNnz)
        return fail(BFS_ERR_INVALID, "bfs_run_csr_noalloc: nnz must lie in [0, " +
                                         std::to_string(bfsk::kStaticMaxNnz) + "] (its scratch is a fixed device array)");
    if (root < 0 || (int64_t)root >= n) return fail(BFS_ERR_INVALID, "root outside [0, n)");
    // the bottom-up scan reads col_ids 16 bytes at a time from 16-byte boundaries of the
    // array, and the offsets are 8-byte loads: a misaligned pointer would fault on the GPU
    if (((uintptr_t)col_ids & 15u) != 0)
        return fail(BFS_ERR_INVALID, "bfs_run_csr_noalloc: col_ids must be 16-byte aligned");
    if (((uintptr_t)row_offsets & 7u) != 0)
        return fail(BFS_ERR_INVALID, "bfs_run_csr_noalloc: row_offsets must be 8-byte aligned");
    if (((uintptr_t)parent_dev & 3u) != 0 || ((uintptr_t)level_dev & 3u) != 0)
        return fail(BFS_ERR_INVALID, "bfs_run_csr_noalloc: parent_dev / level_dev must be 4-byte aligned");
    int dev = 0;
    BFS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(BFS_ERR_UNSUPPORTED, "device index above 63");
    void* base = nullptr;
    int grid = 0;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            // once per device, with that device current: the host-side name of the
            // array is not a device address, so fetch the real one
            void* ptr = nullptr;
            BFS_CUDA_TRY(cudaGetSymbolAddress(&ptr, bfsk::g_noalloc_scratch));
            int sms = 0, occ = 0;
            BFS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            BFS_CUDA_TRY(cudaFuncSetAttribute(bfsk::bfs_single_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)bfsk::kSingleDynSmem));
            BFS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, bfsk::bfs_single_kernel, bfsk::kBlock,
                                                                       bfsk::kSingleDynSmem));
            if (occ < 1) return fail(BFS_ERR_UNSUPPORTED, "BFS kernel cannot be resident on this device");
            g_noalloc_sms[dev] = sms;
            g_noalloc_grid[dev] = occ * sms;
            g_noalloc_ptr[dev] = ptr;
        }
        base = g_noalloc_ptr[dev];
        grid = g_noalloc_grid[dev];
    }
    unsigned char* b = reinterpret_cast<unsigned char*>(base);
    cudaStream_t s = (cudaStream_t)stream;
    const long long W = (n + 31) / 32;
    bfsk::SingleParams p;
    memset(&p, 0, sizeof p);
    p.off = reinterpret_cast<const long long*>(row_offsets);
    p.cols = col_ids;
    p.cols_bu = col_ids;
    p.off_bu = p.off;
    p.isolated = reinterpret_cast<const unsigned*>(b + bfsk::kStaticIsoOff);
    p.n = n;
    p.nnz = nnz;
    p.W = W;
    p.parent = parent_dev;
    p.level = level_dev;
    p.lv8 = nullptr;
    p.visited = reinterpret_cast<unsigned*>(b + bfsk::kStaticVisOff);
    p.front0 = reinterpret_cast<unsigned*>(b + bfsk::kStaticF0Off);
    p.front1 = reinterpret_cast<unsigned*>(b + bfsk::kStaticF1Off);
    p.queue0 = reinterpret_cast<int*>(b + bfsk::kStaticQ0Off);
    p.queue1 = reinterpret_cast<int*>(b + bfsk::kStaticQ1Off);
    p.tasks = reinterpret_cast<bfsk::Task*>(b + bfsk::kStaticTaskOff);
    p.task_cap = bfsk::kStaticTasks;
    p.ctrl = reinterpret_cast<bfsk::Ctrl*>(b + bfsk::kStaticCtrlOff);
    p.rec = reinterpret_cast<bfs_level_record*>(b + bfsk::kStaticRecOff);
    p.rec_cap = bfsk::kStaticRec;
    p.root0 = root;
    p.nroots = 1;
    p.mode = BFS_MODE_DO;
    p.alpha = 14;
    p.beta = 24;
    p.parent_mode = BFS_PARENT_ANY;
    p.big_deg = 96;
    p.td_chunk = bfsk::kChunk;
    p.clu_c = 1;
    p.clu_big = 0;
    p.clu_nf = 0;
    p.clu_mf = 0;
    p.timeout_ns = 10000ull * 1000000ull;
    p.expected = (unsigned)grid;
    const int ig = (int)std::min<long long>((W + 255) / 256, (long long)g_noalloc_sms[dev] * 4);
    bfsk::k_static_isolated<<<ig > 0 ? ig : 1, 256, 0, s>>>(p.off, n, W, const_cast<unsigned*>(p.isolated));
    BFS_CUDA_TRY(cudaGetLastError());
    BFS_CUDA_TRY(cudaMemsetAsync(p.ctrl, 0, sizeof(bfsk::Ctrl), s));
    void* args[] = {&p};
    BFS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)bfsk::bfs_single_kernel, dim3(grid), dim3(bfsk::kBlock),
                                             args, bfsk::kSingleDynSmem, s));
    return BFS_OK;
}
