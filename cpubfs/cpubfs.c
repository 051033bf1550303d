/*
 * cpubfs.c -- multithreaded direction-optimizing BFS on the host cores: the
 * in-node algorithm of Bulu\c{c}, Beamer, Madduri, Asanovic, Patterson,
 * "Distributed-Memory Breadth-First Search on Massive Graphs" (2015), run on one
 * shared-memory node.  A CPU comparator for the benchmark, not part of the GPU
 * library; it shares no code with the CUDA path or with the serial oracle.
 *
 *  top-down step ("Local Computation", top-down): threads split the frontier
 *    queue; each appends newly visited vertices to a thread-local queue, and the
 *    local queues are concatenated into the next frontier at the end of the
 *    level.  The visited check and update are plain loads and stores, not
 *    atomics (the paper's "benign races"): two threads may both claim a vertex
 *    and insert it twice; its level is the same either way and one parent
 *    store wins.  The duplicate insertions are counted.
 *  bottom-up step ("Local Computation", bottom-up; Algorithm 2): threads split
 *    the vertices in 64-vertex words; every vertex not yet completed scans its
 *    row in order and stops at the first neighbour in the current-frontier
 *    bitmap; found vertices go to a separate next-frontier bitmap, each word
 *    written by the one thread that owns it.
 *  direction ("Parallel Direction-Optimizing BFS"): top-down -> bottom-up when
 *    m_f * alpha > m_u, bottom-up -> top-down when n_f * beta < n.
 *  conversions: the next queue is turned into the frontier bitmap (and counted:
 *    distinct vertices vs insertions) before every level; a bottom-up level's
 *    bitmap is turned back into a queue when top-down follows.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t* v;
    int64_t len, cap;
} cb_vec;

static int cb_push(cb_vec* q, int32_t x) {
    if (q->len == q->cap) {
        int64_t nc = q->cap ? 2 * q->cap : 1024;
        int32_t* nv = (int32_t*)realloc(q->v, sizeof(int32_t) * (size_t)nc);
        if (!nv) return -1;
        q->v = nv;
        q->cap = nc;
    }
    q->v[q->len++] = x;
    return 0;
}

/*
 * stats (may be NULL), int64[4]: levels, top-down levels, bottom-up levels,
 * duplicate queue insertions.  Returns the number of levels, or -1 when memory
 * runs out.  threads <= 0: OpenMP's default.
 */
int32_t cb_dobfs(int64_t n, const int64_t* off, const int32_t* cols, int32_t root, int64_t alpha, int64_t beta,
                 int32_t threads, int32_t* parent, int32_t* level, int64_t* stats) {
    if (threads > 0) omp_set_num_threads(threads);
    const int64_t W = (n + 63) / 64;
    const int64_t qcap = 2 * n + 64;   /* insertions of one level, duplicates included */
    uint64_t* front = (uint64_t*)calloc((size_t)W, sizeof(uint64_t));
    uint64_t* next = (uint64_t*)calloc((size_t)W, sizeof(uint64_t));
    uint64_t* done = (uint64_t*)calloc((size_t)W, sizeof(uint64_t));
    int32_t* queue = (int32_t*)malloc(sizeof(int32_t) * (size_t)qcap);
    const int nt = omp_get_max_threads();
    cb_vec* local = (cb_vec*)calloc((size_t)nt, sizeof(cb_vec));
    int64_t* pos = (int64_t*)calloc((size_t)nt + 1, sizeof(int64_t));
    if (!front || !next || !done || !queue || !local || !pos) {
        free(front); free(next); free(done); free(queue); free(local); free(pos);
        return -1;
    }
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; v++) {
        parent[v] = -1;
        level[v] = -1;
    }
    parent[root] = root;
    level[root] = 0;
    done[root >> 6] |= 1ull << (root & 63);
    queue[0] = root;
    int64_t qlen = 1, nf = 1, mf = off[root + 1] - off[root];
    int64_t mu = off[n] - mf, dups = 0, ntd = 0, nbu = 0;
    int prev = 0, d = 0, err = 0;
    int queue_ok = 1, bitmap_ok = 0;   /* which forms of the current frontier are valid */
    while (nf > 0 && !err) {
        const int dir = prev == 0 ? (mf * alpha > mu ? 1 : 0) : (nf * beta < n ? 0 : 1);
        int64_t found = 0, mfound = 0;
        if (dir == 0) {
            ntd++;
            if (!queue_ok) {
                /* bitmap -> queue: per-thread lists of set bits, concatenated in order */
#pragma omp parallel
                {
                    const int t = omp_get_thread_num();
                    local[t].len = 0;
#pragma omp for schedule(static)
                    for (int64_t w = 0; w < W; w++) {
                        uint64_t x = front[w];
                        while (x) {
                            const int b = __builtin_ctzll(x);
                            x &= x - 1;
                            if (cb_push(&local[t], (int32_t)(w * 64 + b))) err = 1;
                        }
                    }
                }
                pos[0] = 0;
                for (int t = 0; t < nt; t++) pos[t + 1] = pos[t] + local[t].len;
#pragma omp parallel for schedule(static)
                for (int t = 0; t < nt; t++) memcpy(queue + pos[t], local[t].v, sizeof(int32_t) * (size_t)local[t].len);
                qlen = pos[nt];
            }
            /* top-down: unsynchronised claims ("benign races": relaxed loads and
               stores, no read-modify-write) into thread-local queues */
#pragma omp parallel
            {
                const int t = omp_get_thread_num();
                local[t].len = 0;
#pragma omp for schedule(dynamic, 64)
                for (int64_t i = 0; i < qlen; i++) {
                    const int32_t u = queue[i];
                    for (int64_t k = off[u]; k < off[u + 1]; k++) {
                        const int32_t v = cols[k];
                        if (__atomic_load_n(&level[v], __ATOMIC_RELAXED) == -1) {
                            __atomic_store_n(&level[v], d + 1, __ATOMIC_RELAXED);
                            __atomic_store_n(&parent[v], u, __ATOMIC_RELAXED);
                            if (cb_push(&local[t], v)) err = 1;
                        }
                    }
                }
            }
            pos[0] = 0;
            for (int t = 0; t < nt; t++) pos[t + 1] = pos[t] + local[t].len;
            if (pos[nt] > qcap) {
                err = 1;
                break;
            }
#pragma omp parallel for schedule(static)
            for (int t = 0; t < nt; t++) memcpy(queue + pos[t], local[t].v, sizeof(int32_t) * (size_t)local[t].len);
            qlen = pos[nt];
            /* the new frontier as a bitmap too, counting its distinct vertices */
            memset(front, 0, sizeof(uint64_t) * (size_t)W);
            int64_t distinct = 0, msum = 0;
#pragma omp parallel for schedule(static) reduction(+ : distinct, msum)
            for (int64_t i = 0; i < qlen; i++) {
                const int32_t v = queue[i];
                const uint64_t bit = 1ull << (v & 63);
                const uint64_t old = __atomic_fetch_or(&front[v >> 6], bit, __ATOMIC_RELAXED);
                if (!(old & bit)) {
                    distinct++;
                    msum += off[v + 1] - off[v];
                }
            }
#pragma omp parallel for schedule(static)
            for (int64_t w = 0; w < W; w++) done[w] |= front[w];
            dups += qlen - distinct;
            found = distinct;
            mfound = msum;
            queue_ok = 1;
            bitmap_ok = 1;
        } else {
            nbu++;
            if (!bitmap_ok) {
                memset(front, 0, sizeof(uint64_t) * (size_t)W);
#pragma omp parallel for schedule(static)
                for (int64_t i = 0; i < qlen; i++)
                    __atomic_fetch_or(&front[queue[i] >> 6], 1ull << (queue[i] & 63), __ATOMIC_RELAXED);
            }
            /* bottom-up (Algorithm 2): each thread owns whole 64-vertex words */
            int64_t fsum = 0, msum = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : fsum, msum)
            for (int64_t w = 0; w < W; w++) {
                uint64_t todo = ~done[w], nx = 0;
                while (todo) {
                    const int b = __builtin_ctzll(todo);
                    todo &= todo - 1;
                    const int64_t u = w * 64 + b;
                    if (u >= n) break;
                    for (int64_t k = off[u]; k < off[u + 1]; k++) {
                        const int32_t v = cols[k];
                        if ((front[v >> 6] >> (v & 63)) & 1ull) {
                            parent[u] = v;
                            level[u] = d + 1;
                            nx |= 1ull << b;
                            fsum++;
                            msum += off[u + 1] - off[u];
                            break;
                        }
                    }
                }
                next[w] = nx;
            }
#pragma omp parallel for schedule(static)
            for (int64_t w = 0; w < W; w++) done[w] |= next[w];
            uint64_t* tmp = front;
            front = next;
            next = tmp;
            found = fsum;
            mfound = msum;
            queue_ok = 0;
            bitmap_ok = 1;
        }
        prev = dir;
        mu -= mfound;
        nf = found;
        mf = mfound;
        d++;
    }
    for (int t = 0; t < nt; t++) free(local[t].v);
    free(front); free(next); free(done); free(queue); free(local); free(pos);
    if (err) return -1;
    if (stats) {
        stats[0] = d;
        stats[1] = ntd;
        stats[2] = nbu;
        stats[3] = dups;
    }
    return d;
}
