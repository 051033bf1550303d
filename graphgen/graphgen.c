/*
 * graphgen.c -- seeded synthetic graph generators (inputs only).
 *
 * These routines produce edge lists and root lists.  They are shared by the
 * CPU oracle tests and the GPU path as *inputs*; nothing here computes any
 * part of the breadth-first search itself (no adjacency build, no frontier,
 * no levels).  Symmetrisation, self-loop removal and de-duplication are left
 * to each consumer (the paper prunes duplicates during preprocessing, see
 * "Data Sets" of Bulu\c{c} et al.), so each side does that on its own.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014).  The i-th output of a
 * generator whose state starts at k is mix(k + (i+1)*gamma), which makes it
 * counter-based: any edge can be generated independently of the others, so
 * the generators below run in parallel threads and still give one fixed
 * result per seed.
 *
 * Graph models:
 *  - R-MAT (Chakrabarti, Zhan, Faloutsos 2004) with initiator (a,b,c,d); the
 *    paper uses a,b,c,d = .57,.19,.19,.05 and edge factor 16 ("Data Sets").
 *    Each of the `scale` recursion levels draws 32 uniform bits and picks a
 *    quadrant by comparing them with integer thresholds round(p * 2^32).
 *    No per-level noise.  This is a Graph500-like stand-in, not the Graph500
 *    reference generator.
 *  - Erdos-Renyi G(n, m): m independent uniform endpoint pairs.
 *  - 2D torus side x side with wrap-around (each vertex linked to its right
 *    and lower neighbour).
 *  - Power-law expected degrees (Chung and Lu, "Connected components in
 *    random graphs with given expected degree sequences", 2002): each edge
 *    end is vertex floor(x) with x drawn from the density proportional to
 *    (x + i0)^(-1/(gamma-1)) on [0, n) by inverting its CDF in closed form,
 *    so vertex rank r has expected degree proportional to (r + i0)^(-1/(gamma-1))
 *    and the degrees follow a power law of exponent gamma.  A scale-free
 *    stand-in for a social graph of a given size (the CDF goes through the
 *    host's libm pow, so one machine always gives one graph per seed).
 * Vertex ids are optionally relabelled by a seeded pseudo-random bijection of
 * [0, n): a few rounds of (odd multiply + add) mod 2^k and xor-shift, each
 * invertible on k-bit integers, with cycle walking when n is not a power of
 * two.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>
#include <unistd.h>

#define GG_GAMMA 0x9E3779B97F4A7C15ULL

static inline uint64_t gg_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* i-th SplitMix64 output of the generator whose state starts at `key`. */
static inline uint64_t gg_rand(uint64_t key, uint64_t i) {
    return gg_mix(key + (i + 1) * GG_GAMMA);
}

/* Independent stream keys derived from (seed, stream id). */
uint64_t gg_stream_key(uint64_t seed, uint64_t stream) {
    return gg_mix(gg_mix(seed) ^ gg_mix(stream * GG_GAMMA + 0x632BE59BD9B4E019ULL));
}

uint64_t gg_splitmix64_output(uint64_t state, uint64_t i) { return gg_rand(state, i); }

/* floor(r * n / 2^64): an unbiased-enough uniform integer in [0, n). */
static inline uint64_t gg_below(uint64_t r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)r * (unsigned __int128)n) >> 64);
}

/* ---------------------------------------------------------------- permutation */

typedef struct {
    uint64_t n, mask;
    int k;
    uint64_t mul[4], add[4];
    int sh[4];
} gg_perm;

static void gg_perm_init(gg_perm* p, uint64_t n, uint64_t seed) {
    p->n = n;
    int k = 0;
    while (k < 63 && ((uint64_t)1 << k) < n) k++;
    p->k = k;
    p->mask = (k == 0) ? 0 : (k >= 64 ? ~0ULL : (((uint64_t)1 << k) - 1));
    uint64_t key = gg_stream_key(seed, 0x7065726dULL);
    for (int r = 0; r < 4; r++) {
        p->mul[r] = gg_rand(key, 2 * r) | 1ULL;
        p->add[r] = gg_rand(key, 2 * r + 1);
        int s = (r & 1) ? (k / 2) : ((k + 1) / 2);
        p->sh[r] = s < 1 ? 1 : s;
    }
}

static inline uint64_t gg_perm_round_trip(const gg_perm* p, uint64_t x) {
    for (int r = 0; r < 4; r++) {
        x = (x * p->mul[r] + p->add[r]) & p->mask;
        x ^= x >> p->sh[r];
    }
    return x;
}

static inline uint64_t gg_perm_apply(const gg_perm* p, uint64_t x) {
    if (p->k == 0) return 0;
    uint64_t y = gg_perm_round_trip(p, x);
    while (y >= p->n) y = gg_perm_round_trip(p, y);  /* cycle walking */
    return y;
}

/* perm_out[i] = image of vertex i under the seeded bijection of [0, n). */
void gg_permutation(int64_t n, uint64_t seed, int32_t* perm_out) {
    gg_perm p;
    gg_perm_init(&p, (uint64_t)n, seed);
    for (int64_t i = 0; i < n; i++) perm_out[i] = (int32_t)gg_perm_apply(&p, (uint64_t)i);
}

/* ---------------------------------------------------------------- threading */

typedef struct {
    int kind;           /* 0 rmat, 1 er, 2 torus, 3 relabel, 4 power law */
    int64_t lo, hi;     /* edge range */
    int scale;
    uint64_t n;
    uint32_t ta, tab, tabc;
    uint64_t key;
    int permute;
    const gg_perm* perm;
    int64_t side;
    double pa, ps, pinv, pi0;   /* power law: i0^b, (n+i0)^b - i0^b, 1/b, i0 */
    int32_t* src;
    int32_t* dst;
} gg_job;

/* one end of a power-law edge: the inverse CDF at the uniform u in [0, 1) */
static inline uint64_t gg_powerlaw_end(const gg_job* j, uint64_t r) {
    const double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);
    double x = pow(u * j->ps + j->pa, j->pinv) - j->pi0;
    if (!(x >= 0.0)) x = 0.0;
    uint64_t id = (uint64_t)x;
    return id < j->n ? id : j->n - 1;
}

static void gg_run_job(gg_job* j) {
    if (j->kind == 0) {
        const int words = (j->scale + 1) / 2;
        for (int64_t i = j->lo; i < j->hi; i++) {
            uint64_t u = 0, v = 0;
            for (int l = 0; l < j->scale; l++) {
                uint64_t w = gg_rand(j->key, (uint64_t)i * (uint64_t)words + (uint64_t)(l >> 1));
                uint32_t r = (l & 1) ? (uint32_t)(w >> 32) : (uint32_t)w;
                uint64_t bu, bv;
                if (r < j->ta)        { bu = 0; bv = 0; }
                else if (r < j->tab)  { bu = 0; bv = 1; }
                else if (r < j->tabc) { bu = 1; bv = 0; }
                else                  { bu = 1; bv = 1; }
                u = (u << 1) | bu;
                v = (v << 1) | bv;
            }
            if (j->permute) { u = gg_perm_apply(j->perm, u); v = gg_perm_apply(j->perm, v); }
            j->src[i] = (int32_t)u;
            j->dst[i] = (int32_t)v;
        }
    } else if (j->kind == 1) {
        for (int64_t i = j->lo; i < j->hi; i++) {
            uint64_t u = gg_below(gg_rand(j->key, 2 * (uint64_t)i), j->n);
            uint64_t v = gg_below(gg_rand(j->key, 2 * (uint64_t)i + 1), j->n);
            if (j->permute) { u = gg_perm_apply(j->perm, u); v = gg_perm_apply(j->perm, v); }
            j->src[i] = (int32_t)u;
            j->dst[i] = (int32_t)v;
        }
    } else if (j->kind == 4) {
        for (int64_t i = j->lo; i < j->hi; i++) {
            uint64_t u = gg_powerlaw_end(j, gg_rand(j->key, 2 * (uint64_t)i));
            uint64_t v = gg_powerlaw_end(j, gg_rand(j->key, 2 * (uint64_t)i + 1));
            if (j->permute) { u = gg_perm_apply(j->perm, u); v = gg_perm_apply(j->perm, v); }
            j->src[i] = (int32_t)u;
            j->dst[i] = (int32_t)v;
        }
    } else if (j->kind == 2) {
        const int64_t s = j->side;
        for (int64_t i = j->lo; i < j->hi; i++) {
            int64_t id = i >> 1, x = id % s, y = id / s;
            int64_t nb = (i & 1) ? (((y + 1) % s) * s + x) : (y * s + (x + 1) % s);
            uint64_t u = (uint64_t)id, v = (uint64_t)nb;
            if (j->permute) { u = gg_perm_apply(j->perm, u); v = gg_perm_apply(j->perm, v); }
            j->src[i] = (int32_t)u;
            j->dst[i] = (int32_t)v;
        }
    }
}

static void* gg_thread_main(void* arg) { gg_run_job((gg_job*)arg); return NULL; }

static int gg_threads(int requested) {
    if (requested > 0) return requested;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    if (c < 1) c = 1;
    if (c > 64) c = 64;
    return (int)c;
}

static void gg_parallel(const gg_job* proto, int64_t m, int nthreads) {
    nthreads = gg_threads(nthreads);
    if (m < 65536) nthreads = 1;
    if (nthreads == 1) { gg_job j = *proto; j.lo = 0; j.hi = m; gg_run_job(&j); return; }
    gg_job* jobs = (gg_job*)malloc(sizeof(gg_job) * (size_t)nthreads);
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    int64_t chunk = (m + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; t++) {
        jobs[t] = *proto;
        jobs[t].lo = (int64_t)t * chunk < m ? (int64_t)t * chunk : m;
        jobs[t].hi = jobs[t].lo + chunk < m ? jobs[t].lo + chunk : m;
        pthread_create(&th[t], NULL, gg_thread_main, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(jobs);
    free(th);
}

/* ---------------------------------------------------------------- generators */

/*
 * R-MAT edge list: m = edgefactor * 2^scale edges in src/dst (caller allocs m
 * each).  Returns 0, or -1 on bad arguments.
 */
int gg_rmat(int scale, int64_t m, double a, double b, double c, uint64_t seed, int permute,
            int32_t* src, int32_t* dst, int nthreads) {
    if (scale < 1 || scale > 30 || m < 0) return -1;
    if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return -1;
    const double two32 = 4294967296.0;
    uint64_t ta = (uint64_t)llround(a * two32);
    uint64_t tab = (uint64_t)llround((a + b) * two32);
    uint64_t tabc = (uint64_t)llround((a + b + c) * two32);
    if (tabc > 0xFFFFFFFFULL) tabc = 0xFFFFFFFFULL;
    if (tab > tabc) tab = tabc;
    if (ta > tab) ta = tab;
    gg_perm perm;
    gg_perm_init(&perm, (uint64_t)1 << scale, seed);
    gg_job j;
    memset(&j, 0, sizeof j);
    j.kind = 0;
    j.scale = scale;
    j.ta = (uint32_t)ta;
    j.tab = (uint32_t)tab;
    j.tabc = (uint32_t)tabc;
    j.key = gg_stream_key(seed, 0x726d6174ULL);
    j.permute = permute;
    j.perm = &perm;
    j.src = src;
    j.dst = dst;
    gg_parallel(&j, m, nthreads);
    return 0;
}

/* Erdos-Renyi G(n, m) edge list (m uniform endpoint pairs).  n <= 2^31-1. */
int gg_er(int64_t n, int64_t m, uint64_t seed, int permute, int32_t* src, int32_t* dst, int nthreads) {
    if (n < 1 || n > 2147483647LL || m < 0) return -1;
    gg_perm perm;
    gg_perm_init(&perm, (uint64_t)n, seed);
    gg_job j;
    memset(&j, 0, sizeof j);
    j.kind = 1;
    j.n = (uint64_t)n;
    j.key = gg_stream_key(seed, 0x6572ULL);
    j.permute = permute;
    j.perm = &perm;
    j.src = src;
    j.dst = dst;
    gg_parallel(&j, m, nthreads);
    return 0;
}

/*
 * Power-law expected-degree graph: m edges, both ends drawn with density
 * proportional to (x + i0)^(-1/(gamma-1)) on [0, n), gamma > 2 (so the
 * exponent 1/(gamma-1) < 1), i0 > 0.  n <= 2^31-1.
 */
int gg_powerlaw(int64_t n, int64_t m, double gamma, double i0, uint64_t seed, int permute, int32_t* src,
                int32_t* dst, int nthreads) {
    if (n < 1 || n > 2147483647LL || m < 0 || !(gamma > 2.0) || !(i0 > 0.0)) return -1;
    const double b = 1.0 - 1.0 / (gamma - 1.0);
    gg_perm perm;
    gg_perm_init(&perm, (uint64_t)n, seed);
    gg_job j;
    memset(&j, 0, sizeof j);
    j.kind = 4;
    j.n = (uint64_t)n;
    j.pi0 = i0;
    j.pa = pow(i0, b);
    j.ps = pow((double)n + i0, b) - j.pa;
    j.pinv = 1.0 / b;
    j.key = gg_stream_key(seed, 0x706c6177ULL);
    j.permute = permute;
    j.perm = &perm;
    j.src = src;
    j.dst = dst;
    gg_parallel(&j, m, nthreads);
    return 0;
}

/* side x side torus: 2*side^2 edges (right and lower neighbour, wrapping). */
int gg_torus(int64_t side, uint64_t seed, int permute, int32_t* src, int32_t* dst, int nthreads) {
    if (side < 1 || side * side > 2147483647LL) return -1;
    gg_perm perm;
    gg_perm_init(&perm, (uint64_t)(side * side), seed);
    gg_job j;
    memset(&j, 0, sizeof j);
    j.kind = 2;
    j.side = side;
    j.permute = permute;
    j.perm = &perm;
    j.src = src;
    j.dst = dst;
    gg_parallel(&j, 2 * side * side, nthreads);
    return 0;
}

/*
 * Pick k distinct roots uniformly among vertices that are an endpoint of at
 * least one edge whose two ends differ (i.e. vertices that keep degree > 0
 * after self-loops are dropped).  Returns the number of roots written
 * (< k only if fewer candidates exist), or -1 on bad ids.
 */
int64_t gg_pick_roots(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int64_t k,
                      uint64_t seed, int32_t* roots) {
    uint8_t* mark = (uint8_t*)calloc((size_t)n, 1);
    if (!mark) return -1;
    for (int64_t i = 0; i < m; i++) {
        int32_t u = src[i], v = dst[i];
        if (u < 0 || v < 0 || u >= n || v >= n) { free(mark); return -1; }
        if (u != v) { mark[u] = 1; mark[v] = 1; }
    }
    int64_t cnt = 0;
    for (int64_t v = 0; v < n; v++) cnt += mark[v];
    int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cnt > 0 ? cnt : 1));
    if (!cand) { free(mark); return -1; }
    int64_t p = 0;
    for (int64_t v = 0; v < n; v++) if (mark[v]) cand[p++] = (int32_t)v;
    free(mark);
    uint64_t key = gg_stream_key(seed, 0x726f6f74ULL);
    int64_t take = k < cnt ? k : cnt;
    for (int64_t j = 0; j < take; j++) {  /* partial Fisher-Yates */
        int64_t r = j + (int64_t)gg_below(gg_rand(key, (uint64_t)j), (uint64_t)(cnt - j));
        int32_t t = cand[j];
        cand[j] = cand[r];
        cand[r] = t;
        roots[j] = cand[j];
    }
    free(cand);
    return take;
}
