/*
 * oracle.c -- serial CPU oracle for level-synchronous breadth-first search.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or table with the CUDA path, and the CUDA path never calls it.
 *
 * Plain, slow, obviously correct C.  Each routine cites the passage of
 * Bulu\c{c}, Beamer, Madduri, Asanovic, Patterson, "Distributed-Memory
 * Breadth-First Search on Massive Graphs" (2015) that it follows:
 *
 *  (the CSR itself is built by the Python side of the oracle with numpy's
 *  sort, as the set definition of "Graph Representation" / "Data Sets")
 *  or_bfs_topdown    Algorithm 1 (sequential top-down BFS), FIFO queue, with
 *                    the hop count d of the "Breadth-First Search" section
 *                    recorded alongside the parent.
 *  or_bfs_bottomup   Algorithm 2 (sequential bottom-up BFS): every unvisited
 *                    vertex scans its neighbours for one in the *current*
 *                    frontier and stops at the first; the next frontier is
 *                    separate and swapped in at the end of the level.
 *  or_min_parent     the (select2nd, min) semiring of the parallel top-down
 *                    algorithm's local discovery: among the valid parents the
 *                    minimum id.
 *  or_components     union-find connected components (independent of BFS),
 *                    used to check that the reached set is the component of
 *                    the root ("examines the whole connected component").
 *  or_certify        the invariants that make a level/parent pair a BFS:
 *                    see the function comment.
 *  or_do_schedule    the direction-optimizing schedule ("Parallel
 *                    Direction-Optimizing BFS"): per level the direction chosen
 *                    by the edges-out-of-frontier / frontier-size heuristics,
 *                    and the per-level work counts that the byte model uses.
 *  or_do_schedule_dir the same schedule on a directed graph (top-down over
 *                    out-edges, bottom-up over in-edges: "Data Sets" says the
 *                    method applies to directed graphs, and the bottom-up step
 *                    needs the transpose, "Data Decomposition").
 *  or_reach          depth-first reachability (the reached set, independently).
 *  or_certify_dir    the BFS invariants along directed edges.
 *  or_hub_first      the rows in the order a bottom-up step may scan them:
 *                    neighbours by degree, highest first, ties by id (Algorithm
 *                    2 fixes no order beyond "in order"); each row sorted on
 *                    its own, for graphs too large for the numpy lexsort.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ Algorithm 1 */

/*
 * Sequential top-down BFS (Algorithm 1).  parent[v] = -1 unless reached,
 * parent[root] = root; level[v] = hop distance (-1 if unreachable).
 * `queue` is scratch of n entries.  Returns the number of levels (the
 * largest level + 1).  Ties among parents go to the first discoverer in FIFO
 * order.
 */
int32_t or_bfs_topdown(int64_t n, const int64_t* off, const int32_t* cols, int32_t root,
                       int32_t* parent, int32_t* level, int32_t* queue) {
    for (int64_t v = 0; v < n; v++) { parent[v] = -1; level[v] = -1; }
    parent[root] = root;
    level[root] = 0;
    /* frontier = queue[head, mid), next = queue[mid, tail): one FIFO holds both */
    int64_t head = 0, tail = 0;
    queue[tail++] = root;
    int32_t d = 0;
    while (head < tail) {                      /* while frontier != empty */
        int64_t mid = tail;
        for (; head < mid; head++) {           /* for each u in frontier */
            int32_t u = queue[head];
            for (int64_t k = off[u]; k < off[u + 1]; k++) {  /* each neighbour v */
                int32_t v = cols[k];
                if (parent[v] == -1) {         /* unvisited */
                    queue[tail++] = v;         /* next <- next + {v} */
                    parent[v] = u;
                    level[v] = d + 1;
                }
            }
        }
        d++;                                   /* frontier <- next */
    }
    return d;
}

/* ------------------------------------------------------------------ Algorithm 2 */

/*
 * Sequential bottom-up BFS (Algorithm 2).  Same outputs as or_bfs_topdown.
 * frontier/next are scratch byte arrays of n entries.  Membership is tested
 * against the current frontier only; `next` becomes the frontier after the
 * whole level.  Returns the number of levels.
 */
int32_t or_bfs_bottomup(int64_t n, const int64_t* off, const int32_t* cols, int32_t root,
                        int32_t* parent, int32_t* level, uint8_t* frontier, uint8_t* next) {
    for (int64_t v = 0; v < n; v++) { parent[v] = -1; level[v] = -1; frontier[v] = 0; next[v] = 0; }
    parent[root] = root;
    level[root] = 0;
    frontier[root] = 1;
    int64_t fsize = 1;
    int32_t d = 0;
    while (fsize > 0) {
        int64_t nsize = 0;
        for (int64_t u = 0; u < n; u++) {
            if (parent[u] != -1) continue;     /* only unvisited vertices search */
            for (int64_t k = off[u]; k < off[u + 1]; k++) {
                int32_t v = cols[k];
                if (frontier[v]) {
                    next[u] = 1;
                    parent[u] = v;
                    level[u] = d + 1;
                    nsize++;
                    break;                     /* early exit */
                }
            }
        }
        uint8_t* t = frontier; frontier = next; next = t;   /* frontier <- next */
        for (int64_t v = 0; v < n; v++) next[v] = 0;
        fsize = nsize;
        d++;
    }
    return d;
}

/* ------------------------------------------------------------------ min-id parent */

/* parent[v] = min{u in adj(v) : level[u] = level[v]-1}; parent[root] = root; -1 if unreached. */
void or_min_parent(int64_t n, const int64_t* off, const int32_t* cols, const int32_t* level,
                   int32_t* parent) {
    for (int64_t v = 0; v < n; v++) {
        parent[v] = -1;
        if (level[v] == 0) { parent[v] = (int32_t)v; continue; }
        if (level[v] < 0) continue;
        for (int64_t k = off[v]; k < off[v + 1]; k++) {
            int32_t u = cols[k];
            if (level[u] == level[v] - 1 && (parent[v] == -1 || u < parent[v])) parent[v] = u;
        }
    }
}

/* ------------------------------------------------------------------ union-find */

static int32_t or_find(int32_t* p, int32_t x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }   /* path halving */
    return x;
}

/* label[v] = smallest vertex id of v's connected component. */
void or_components(int64_t n, const int64_t* off, const int32_t* cols, int32_t* label) {
    for (int64_t v = 0; v < n; v++) label[v] = (int32_t)v;
    for (int64_t u = 0; u < n; u++)
        for (int64_t k = off[u]; k < off[u + 1]; k++) {
            int32_t a = or_find(label, (int32_t)u), b = or_find(label, cols[k]);
            if (a != b) { if (a < b) label[b] = a; else label[a] = b; }
        }
    for (int64_t v = 0; v < n; v++) label[v] = or_find(label, (int32_t)v);
}

/* ------------------------------------------------------------------ certificate */

/* binary search for v in the sorted row u */
static int or_has_edge(const int64_t* off, const int32_t* cols, int32_t u, int32_t v) {
    int64_t lo = off[u], hi = off[u + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (cols[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo < off[u + 1] && cols[lo] == v;
}

/*
 * Check that (level, parent) is a breadth-first search from `root`:
 *   1 level[root] = 0 and parent[root] = root (when parent is given)
 *   2 for every reached v != root: level[v] >= 1, (parent[v], v) is an edge,
 *     level[parent[v]] = level[v] - 1
 *   3 every edge {u, v} with both ends reached spans at most one level
 *   4 an edge never joins a reached and an unreached vertex
 *   5 the reached set is exactly the connected component of root (label[]
 *     from or_components) and unreached vertices carry parent = level = -1.
 * 2 gives dist <= level along the parent chain; 3 gives level <= dist along a
 * shortest path; together level = dist.  `parent` may be NULL: then 2 asks
 * instead that every reached v != root has some neighbour at level[v] - 1 and
 * that only the root sits at level 0, which gives the same chain (dist <=
 * level) without naming the parents.  Returns 0 if valid, else
 * (code << 40) | vertex where code is the failed invariant.
 */
int64_t or_certify(int64_t n, const int64_t* off, const int32_t* cols, int32_t root,
                   const int32_t* parent, const int32_t* level, const int32_t* label) {
    if (root < 0 || root >= n) return (int64_t)1 << 40;
    if (level[root] != 0) return ((int64_t)1 << 40) | root;
    if (parent && parent[root] != root) return ((int64_t)1 << 40) | root;
    for (int64_t v = 0; v < n; v++) {
        int reached = level[v] >= 0;
        int in_comp = label[v] == label[root];
        if (reached != in_comp) return ((int64_t)5 << 40) | v;
        if (!reached) {
            if (level[v] != -1 || (parent && parent[v] != -1)) return ((int64_t)5 << 40) | v;
            continue;
        }
        if (v != root) {
            if (level[v] < 1) return ((int64_t)2 << 40) | v;
            if (parent) {
                int32_t p = parent[v];
                if (p < 0 || p >= n) return ((int64_t)2 << 40) | v;
                if (!or_has_edge(off, cols, p, (int32_t)v)) return ((int64_t)2 << 40) | v;
                if (level[p] != level[v] - 1) return ((int64_t)2 << 40) | v;
            } else {
                int has_pred = 0;
                for (int64_t k = off[v]; k < off[v + 1] && !has_pred; k++)
                    if (level[cols[k]] == level[v] - 1) has_pred = 1;
                if (!has_pred) return ((int64_t)2 << 40) | v;
            }
        }
        for (int64_t k = off[v]; k < off[v + 1]; k++) {
            int32_t u = cols[k];
            if (level[u] < 0) return ((int64_t)4 << 40) | v;
            int32_t diff = level[u] - level[v];
            if (diff > 1 || diff < -1) return ((int64_t)3 << 40) | v;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ DO schedule */

/*
 * Direction-optimizing schedule from the exact levels.  The paper chooses,
 * per level, top-down or bottom-up by "the number of edges originating in the
 * frontier while top-down and the size of the frontier while bottom-up".  With
 * the thresholds alpha, beta the rule read here is:
 *   in top-down:  go bottom-up when m_f * alpha > m_u
 *   in bottom-up: go top-down  when n_f * beta  < n
 * where, at the start of level d, n_f = |frontier| = |{v : level[v] = d}|,
 * m_f = sum of degrees over the frontier, m_u = sum of degrees over vertices
 * not yet reached (level > d or unreachable).  The first level starts from
 * top-down and is itself subject to the rule.  mode: 0 = direction-optimizing,
 * 1 = top-down only, 2 = bottom-up only.
 *
 * Per level d (d < num_levels) the arrays receive:
 *   dir[d]      0 top-down, 1 bottom-up
 *   nf[d], mf[d]       frontier size and degree sum
 *   nnext[d]    vertices discovered (|{v : level[v] = d+1}|)
 *   mnext[d]    their degree sum
 *   scanned[d]  bottom-up only: unvisited vertices with degree > 0 that search
 *   examined[d] top-down: m_f; bottom-up: sum over searching vertices of the
 *               1-based position of the first frontier neighbour in sorted
 *               order, or the degree if none (the serial early-exit count)
 * Returns num_levels, or -1 if cap is too small.
 */
int32_t or_do_schedule_dir(int64_t n, const int64_t* off_out, const int64_t* off_bu, const int32_t* cols_bu,
                           const int32_t* level, int32_t mode, int64_t alpha, int64_t beta, int32_t cap,
                           int32_t* dir, int64_t* nf, int64_t* mf, int64_t* nnext, int64_t* mnext,
                           int64_t* scanned, int64_t* examined);

int32_t or_do_schedule(int64_t n, const int64_t* off, const int32_t* cols, const int32_t* level,
                       int32_t mode, int64_t alpha, int64_t beta, int32_t cap,
                       int32_t* dir, int64_t* nf, int64_t* mf, int64_t* nnext, int64_t* mnext,
                       int64_t* scanned, int64_t* examined) {
    return or_do_schedule_dir(n, off, off, cols, level, mode, alpha, beta, cap, dir, nf, mf, nnext, mnext,
                              scanned, examined);
}

/*
 * The same schedule on a directed graph: a top-down step expands the
 * frontier's out-edges (off_out), a bottom-up step lets an unvisited vertex
 * scan its in-edges (the transpose: off_bu, cols_bu), so m_f = sum of
 * out-degrees over the frontier and m_u = sum of in-degrees over the vertices
 * not yet reached (the edges a bottom-up step could still examine); scanned
 * counts unvisited vertices with in-degree > 0; mnext is the out-degree sum
 * of the next frontier.  With off_out == off_bu (an undirected graph) this is
 * or_do_schedule.
 */
int32_t or_do_schedule_dir(int64_t n, const int64_t* off_out, const int64_t* off_bu, const int32_t* cols_bu,
                           const int32_t* level, int32_t mode, int64_t alpha, int64_t beta, int32_t cap,
                           int32_t* dir, int64_t* nf, int64_t* mf, int64_t* nnext, int64_t* mnext,
                           int64_t* scanned, int64_t* examined) {
    int32_t L = 0;
    for (int64_t v = 0; v < n; v++) if (level[v] + 1 > L) L = level[v] + 1;
    if (L > cap) return -1;
    int64_t* cnt = (int64_t*)calloc((size_t)L + 1, sizeof(int64_t));
    int64_t* deg = (int64_t*)calloc((size_t)L + 1, sizeof(int64_t));     /* out-degree sum per level */
    int64_t* ideg = (int64_t*)calloc((size_t)L + 1, sizeof(int64_t));    /* in-degree sum per level */
    int64_t nnz_in = off_bu[n];
    for (int64_t v = 0; v < n; v++) {
        if (level[v] >= 0) {
            cnt[level[v]]++;
            deg[level[v]] += off_out[v + 1] - off_out[v];
            ideg[level[v]] += off_bu[v + 1] - off_bu[v];
        }
    }
    int64_t m_u = nnz_in - ideg[0];   /* in-degree sum of vertices not in levels 0..d */
    int32_t cur = 0;                  /* start top-down */
    for (int32_t d = 0; d < L; d++) {
        int64_t n_f = cnt[d], m_f = deg[d];
        if (mode == 1) cur = 0;
        else if (mode == 2) cur = 1;
        else if (cur == 0 && m_f * alpha > m_u) cur = 1;
        else if (cur == 1 && n_f * beta < n) cur = 0;
        dir[d] = cur;
        nf[d] = n_f;
        mf[d] = m_f;
        nnext[d] = cnt[d + 1];
        mnext[d] = deg[d + 1];
        if (cur == 0) {
            scanned[d] = 0;
            examined[d] = m_f;
        } else {
            int64_t sc = 0, ex = 0;
            for (int64_t u = 0; u < n; u++) {
                if (level[u] >= 0 && level[u] <= d) continue;   /* already visited */
                int64_t b = off_bu[u], e = off_bu[u + 1];
                if (e == b) continue;                          /* no in-edge: never searches */
                sc++;
                int64_t pos = e - b;
                for (int64_t k = b; k < e; k++)
                    if (level[cols_bu[k]] == d) { pos = k - b + 1; break; }
                ex += pos;
            }
            scanned[d] = sc;
            examined[d] = ex;
        }
        m_u -= ideg[d + 1];
    }
    free(cnt);
    free(deg);
    free(ideg);
    return L;
}

/* ------------------------------------------------------------------ directed graphs */

/*
 * Vertices reachable from root along out-edges, by an explicit-stack depth-
 * first search (a different traversal order from breadth-first search, used
 * to check the reached set independently).  mark[v] = 1 if reachable.
 * Returns the number reached, or -1 if scratch memory could not be allocated.
 */
int64_t or_reach(int64_t n, const int64_t* off, const int32_t* cols, int32_t root, uint8_t* mark) {
    int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!stack) return -1;
    for (int64_t v = 0; v < n; v++) mark[v] = 0;
    int64_t top = 0, cnt = 1;
    stack[top++] = root;
    mark[root] = 1;
    while (top > 0) {
        int32_t u = stack[--top];
        for (int64_t k = off[u]; k < off[u + 1]; k++) {
            int32_t v = cols[k];
            if (!mark[v]) {
                mark[v] = 1;
                cnt++;
                stack[top++] = v;
            }
        }
    }
    free(stack);
    return cnt;
}

/*
 * Check that (level, parent) is a breadth-first search from root along the
 * out-edges of a directed graph (off/cols = the out-edge CSR):
 *   1 level[root] = 0 and parent[root] = root (when parent is given)
 *   2 for every reached v != root: level[v] >= 1, (parent[v] -> v) is an edge,
 *     level[parent[v]] = level[v] - 1 (without parents: some in-neighbour of v
 *     sits at level[v] - 1, found by scanning the out-rows of all vertices)
 *   3 every edge u -> v out of a reached u ends at a reached v with
 *     level[v] <= level[u] + 1
 *   4 (unused code, kept apart from the undirected checker's numbering)
 *   5 the reached set is exactly reach[] (or_reach) and unreached vertices
 *     carry parent = level = -1.
 * 2 gives dist <= level along the parent chain, 3 gives level <= dist along a
 * shortest directed path; together level = dist.  Returns 0 if valid, else
 * (code << 40) | vertex.
 */
int64_t or_certify_dir(int64_t n, const int64_t* off, const int32_t* cols, int32_t root, const int32_t* parent,
                       const int32_t* level, const uint8_t* reach) {
    if (root < 0 || root >= n) return (int64_t)1 << 40;
    if (level[root] != 0) return ((int64_t)1 << 40) | root;
    if (parent && parent[root] != root) return ((int64_t)1 << 40) | root;
    uint8_t* has_pred = NULL;
    if (!parent) {
        has_pred = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
        if (!has_pred) return ((int64_t)6 << 40);
        for (int64_t u = 0; u < n; u++) {
            if (level[u] < 0) continue;
            for (int64_t k = off[u]; k < off[u + 1]; k++)
                if (level[cols[k]] == level[u] + 1) has_pred[cols[k]] = 1;
        }
    }
    int64_t bad = 0;
    for (int64_t v = 0; v < n && !bad; v++) {
        int reached = level[v] >= 0;
        if (reached != (reach[v] != 0)) { bad = ((int64_t)5 << 40) | v; break; }
        if (!reached) {
            if (level[v] != -1 || (parent && parent[v] != -1)) bad = ((int64_t)5 << 40) | v;
            continue;
        }
        if (v != root) {
            if (level[v] < 1) { bad = ((int64_t)2 << 40) | v; break; }
            if (parent) {
                int32_t p = parent[v];
                if (p < 0 || p >= n || !or_has_edge(off, cols, p, (int32_t)v) || level[p] != level[v] - 1) {
                    bad = ((int64_t)2 << 40) | v;
                    break;
                }
            } else if (!has_pred[v]) {
                bad = ((int64_t)2 << 40) | v;
                break;
            }
        }
        for (int64_t k = off[v]; k < off[v + 1]; k++) {
            int32_t u = cols[k];
            if (level[u] < 0 || level[u] > level[v] + 1) { bad = ((int64_t)3 << 40) | v; break; }
        }
    }
    free(has_pred);
    return bad;
}

/* ------------------------------------------------------------------ hub-first rows */

/*
 * Rows u0 <= u < u1 of out = the column ids with every row reordered by
 * (degree descending, id ascending), the same rows in the same place (offsets
 * unchanged, indices absolute).  Each row is sorted on its own with the key
 * (~degree << 32) | id, which orders by degree descending and then id
 * ascending (ids are unique within a row): insertion sort for short rows, a
 * bottom-up merge sort for long ones.  Disjoint row ranges may run in
 * parallel.  Returns 0, or -1 if scratch memory could not be allocated.
 */
static uint64_t or_hub_key(const int64_t* off, int32_t v) {
    uint64_t d = (uint64_t)(off[v + 1] - off[v]);
    if (d > 0xFFFFFFFFull) d = 0xFFFFFFFFull;
    return ((0xFFFFFFFFull - d) << 32) | (uint32_t)v;
}

int32_t or_hub_first(int64_t n, const int64_t* off, const int32_t* cols, int32_t* out, int64_t u0, int64_t u1) {
    (void)n;
    int64_t maxdeg = 0;
    for (int64_t u = u0; u < u1; u++)
        if (off[u + 1] - off[u] > maxdeg) maxdeg = off[u + 1] - off[u];
    uint64_t* a = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(maxdeg > 0 ? maxdeg : 1));
    uint64_t* b = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(maxdeg > 0 ? maxdeg : 1));
    if (!a || !b) {
        free(a);
        free(b);
        return -1;
    }
    for (int64_t u = u0; u < u1; u++) {
        const int64_t s = off[u], len = off[u + 1] - s;
        for (int64_t k = 0; k < len; k++) a[k] = or_hub_key(off, cols[s + k]);
        if (len <= 32) {
            for (int64_t i = 1; i < len; i++) {
                uint64_t x = a[i];
                int64_t j = i - 1;
                while (j >= 0 && a[j] > x) {
                    a[j + 1] = a[j];
                    j--;
                }
                a[j + 1] = x;
            }
        } else {
            /* bottom-up merge sort, runs of width 1, 2, 4, ... alternating a and b */
            uint64_t* src = a;
            uint64_t* dst = b;
            for (int64_t wdt = 1; wdt < len; wdt *= 2) {
                for (int64_t lo = 0; lo < len; lo += 2 * wdt) {
                    int64_t mid = lo + wdt < len ? lo + wdt : len;
                    int64_t hi = lo + 2 * wdt < len ? lo + 2 * wdt : len;
                    int64_t i = lo, j = mid, k = lo;
                    while (i < mid && j < hi) dst[k++] = src[i] <= src[j] ? src[i++] : src[j++];
                    while (i < mid) dst[k++] = src[i++];
                    while (j < hi) dst[k++] = src[j++];
                }
                uint64_t* t = src;
                src = dst;
                dst = t;
            }
            if (src != a) memcpy(a, src, sizeof(uint64_t) * (size_t)len);
        }
        for (int64_t k = 0; k < len; k++) out[s + k] = (int32_t)(uint32_t)(a[k] & 0xFFFFFFFFull);
    }
    free(a);
    free(b);
    return 0;
}
