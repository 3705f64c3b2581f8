/*
 * gen.c -- seeded synthetic inputs shared by the oracle side and the CUDA side.
 *
 * This module holds no shortest-path or priority-queue arithmetic.  It only
 * draws graphs (CSR arrays) and heap update batches from a counter-based
 * pseudo-random stream, so that the oracle and the GPU path can be fed the
 * same inputs without sharing any of the method's code.
 *
 * Random stream: SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014), in the 64-bit finaliser form
 * popularised by Vigna.  Bounded integers are drawn by rejection of the
 * incomplete top bucket, so they are exactly uniform.  Distinct samples use
 * Floyd's algorithm (Bentley and Floyd, "Programming Pearls: A sample of
 * brilliance", CACM 1987).
 *
 * CSR layout everywhere: row_ptr u64[n+1], col u32[m], w u32[m]; the targets
 * of one vertex are stored in ascending order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- stream */

static inline uint64_t sm64_next(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Uniform integer in [lo, hi] (inclusive), rejection sampling. */
static inline uint64_t sm64_range(uint64_t *s, uint64_t lo, uint64_t hi)
{
    uint64_t span = hi - lo;
    if (span == UINT64_MAX)
        return sm64_next(s);
    uint64_t range = span + 1;
    uint64_t rem = (UINT64_MAX % range + 1) % range; /* 2^64 mod range */
    uint64_t x;
    if (rem == 0)
        return lo + sm64_next(s) % range;
    uint64_t limit = (uint64_t)0 - rem; /* largest multiple of range, mod 2^64 */
    do {
        x = sm64_next(s);
    } while (x >= limit);
    return lo + x % range;
}

/* Independent sub-streams of one seed: one for structure, one for weights. */
static uint64_t stream_seed(uint64_t seed, uint64_t tag)
{
    uint64_t s = seed ^ (tag * 0xD1B54A32D192ED03ULL);
    return sm64_next(&s);
}

uint64_t gen_splitmix64(uint64_t *state) { return sm64_next(state); }

uint64_t gen_uniform(uint64_t *state, uint64_t lo, uint64_t hi)
{
    return sm64_range(state, lo, hi);
}

/* Fill out[0..count) with uniform integers in [lo, hi]. */
void gen_uniform_array_u32(uint64_t seed, uint32_t lo, uint32_t hi, uint32_t *out, uint64_t count)
{
    uint64_t s = stream_seed(seed, 7);
    for (uint64_t i = 0; i < count; i++)
        out[i] = (uint32_t)sm64_range(&s, lo, hi);
}

static void draw_weights(uint64_t seed, uint32_t wlo, uint32_t whi, uint32_t *w, uint64_t m)
{
    uint64_t s = stream_seed(seed, 2);
    for (uint64_t e = 0; e < m; e++)
        w[e] = (uint32_t)sm64_range(&s, wlo, whi);
}

static int cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------ grid graph */

/* Number of arcs of a rows x cols 4-neighbour directed grid. */
uint64_t gen_grid_edges(uint32_t rows, uint32_t cols)
{
    uint64_t r = rows, c = cols;
    return 4 * r * c - 2 * r - 2 * c;
}

/*
 * rows x cols grid, vertex id = row * cols + col (row-major).  Every vertex has
 * one directed arc to each existing neighbour (up, left, right, down, which is
 * ascending target order), each arc with its own weight drawn uniformly in
 * [wlo, whi] in CSR order.
 */
void gen_grid(uint32_t rows, uint32_t cols, uint32_t wlo, uint32_t whi, uint64_t seed,
              uint64_t *row_ptr, uint32_t *col, uint32_t *w)
{
    uint64_t e = 0;
    for (uint32_t r = 0; r < rows; r++) {
        for (uint32_t c = 0; c < cols; c++) {
            uint32_t v = r * cols + c;
            row_ptr[v] = e;
            if (r > 0) col[e++] = v - cols;
            if (c > 0) col[e++] = v - 1;
            if (c + 1 < cols) col[e++] = v + 1;
            if (r + 1 < rows) col[e++] = v + cols;
        }
    }
    row_ptr[(uint64_t)rows * cols] = e;
    draw_weights(seed, wlo, whi, w, e);
}

/* ---------------------------------------------------------- banded graph */

static uint32_t banded_candidates(uint32_t n, uint32_t i, uint32_t win, uint32_t *lo_out)
{
    uint32_t lo = i > win ? i - win : 0;
    uint64_t hi = (uint64_t)i + win;
    if (hi > (uint64_t)n - 1) hi = n - 1;
    *lo_out = lo;
    return (uint32_t)(hi - lo + 1) - 1; /* vertex i itself is excluded */
}

/* Exact edge count of gen_banded for these parameters. */
uint64_t gen_banded_edges(uint32_t n, uint32_t deg, uint32_t win)
{
    uint64_t m = 0;
    for (uint32_t i = 0; i < n; i++) {
        uint32_t lo, cnt = banded_candidates(n, i, win, &lo);
        m += cnt < deg ? cnt : deg;
    }
    return m;
}

/*
 * Banded high-diameter graph: vertex i has min(deg, #candidates) out-arcs to
 * distinct vertices drawn uniformly from [i - win, i + win] clipped to
 * [0, n - 1], excluding i.  Targets of each vertex sorted ascending.  Weights
 * uniform in [wlo, whi], drawn in CSR order from a second stream.
 */
void gen_banded(uint32_t n, uint32_t deg, uint32_t win, uint32_t wlo, uint32_t whi, uint64_t seed,
                uint64_t *row_ptr, uint32_t *col, uint32_t *w)
{
    uint64_t s = stream_seed(seed, 1);
    uint64_t e = 0;
    uint64_t span = 2 * (uint64_t)win + 1;
    uint32_t *pick = (uint32_t *)malloc(sizeof(uint32_t) * (deg ? deg : 1));
    uint32_t *mark = (uint32_t *)calloc(span, sizeof(uint32_t)); /* index -> i+1 if picked */
    for (uint32_t i = 0; i < n; i++) {
        uint32_t lo, cnt = banded_candidates(n, i, win, &lo);
        uint32_t k = cnt < deg ? cnt : deg;
        /* Floyd: k distinct indices out of [0, cnt) */
        uint32_t np = 0;
        for (uint32_t j = cnt - k; j < cnt; j++) {
            uint32_t t = (uint32_t)sm64_range(&s, 0, j);
            uint32_t x = mark[t] == i + 1 ? j : t;
            mark[x] = i + 1;
            pick[np++] = x;
        }
        for (uint32_t q = 0; q < np; q++) {
            uint32_t v = lo + pick[q];
            if (v >= i) v += 1; /* skip the vertex itself */
            pick[q] = v;
        }
        qsort(pick, np, sizeof(uint32_t), cmp_u32);
        row_ptr[i] = e;
        memcpy(col + e, pick, sizeof(uint32_t) * np);
        e += np;
    }
    row_ptr[n] = e;
    free(pick);
    free(mark);
    draw_weights(seed, wlo, whi, w, e);
}

/* ------------------------------------------------- random (test) graph */

/*
 * m arcs with endpoints uniform in [0, n) (self-loops and parallel arcs
 * allowed), stored in CSR by source; arcs keep their draw order within a
 * source.  Used for small randomized tests.
 */
void gen_random_graph(uint32_t n, uint64_t m, uint32_t wlo, uint32_t whi, uint64_t seed,
                      uint64_t *row_ptr, uint32_t *col, uint32_t *w)
{
    uint64_t s = stream_seed(seed, 3);
    uint32_t *src = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t *dst = (uint32_t *)malloc(sizeof(uint32_t) * (m ? m : 1));
    for (uint64_t e = 0; e < m; e++) {
        src[e] = (uint32_t)sm64_range(&s, 0, n - 1);
        dst[e] = (uint32_t)sm64_range(&s, 0, n - 1);
    }
    memset(row_ptr, 0, sizeof(uint64_t) * ((uint64_t)n + 1));
    for (uint64_t e = 0; e < m; e++) row_ptr[src[e] + 1]++;
    for (uint32_t v = 0; v < n; v++) row_ptr[v + 1] += row_ptr[v];
    uint64_t *fill = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    memcpy(fill, row_ptr, sizeof(uint64_t) * n);
    for (uint64_t e = 0; e < m; e++) col[fill[src[e]]++] = dst[e];
    free(fill);
    free(src);
    free(dst);
    draw_weights(seed, wlo, whi, w, m);
}

/* ----------------------------------------------- the paper's random DAG */

/*
 * Random DAG of the paper's experiments (Section 4.2), 0-indexed: the chain
 * (i, i+1) with weight 1 for every i < n - 1, plus extra forward arcs (u, v),
 * u < v, v != u + 1, each with weight 2 * (v - u) so that the chain stays the
 * unique shortest path.  The extra arcs are spread as evenly as possible over
 * the sources 0 .. n - 2 (water-filling: vertex u can take at most n - u - 2
 * extra arcs), and the targets of one source are distinct and uniform.
 * deg_out[u] receives the out-degree of u; the caller sizes the arrays from
 * gen_dag_degrees() first.
 */
uint64_t gen_dag_degrees(uint32_t n, uint64_t m, uint64_t *deg_out)
{
    if (n == 0) return 0;
    uint64_t chain = n - 1;
    uint64_t extra = m > chain ? m - chain : 0;
    for (uint32_t u = 0; u < n; u++) deg_out[u] = 0;
    /* water-fill: repeatedly give every unsaturated source an equal share */
    uint64_t left = extra;
    uint32_t active = n >= 2 ? n - 1 : 0; /* sources 0..n-2 */
    while (left > 0 && active > 0) {
        uint64_t share = left / active;
        if (share == 0) share = 1;
        uint32_t still = 0;
        for (uint32_t u = 0; u + 1 < n && left > 0; u++) {
            uint64_t cap = (uint64_t)(n - u - 2);
            if (deg_out[u] >= cap) continue;
            uint64_t give = cap - deg_out[u];
            if (give > share) give = share;
            if (give > left) give = left;
            deg_out[u] += give;
            left -= give;
            if (deg_out[u] < cap) still++;
        }
        active = still;
    }
    uint64_t total = 0;
    for (uint32_t u = 0; u + 1 < n; u++) {
        deg_out[u] += 1; /* the chain arc */
        total += deg_out[u];
    }
    return total;
}

void gen_dag(uint32_t n, uint64_t m, uint64_t seed, uint64_t *row_ptr, uint32_t *col, uint32_t *w)
{
    uint64_t *deg = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    gen_dag_degrees(n, m, deg);
    uint64_t s = stream_seed(seed, 4);
    uint64_t e = 0;
    uint32_t *mark = (uint32_t *)calloc(n ? n : 1, sizeof(uint32_t)); /* index -> u+1 if picked */
    uint32_t *pick = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    for (uint32_t u = 0; u < n; u++) {
        row_ptr[u] = e;
        if (deg[u] == 0) continue;
        uint64_t k = deg[u] - 1;              /* extra arcs */
        uint64_t cnt = (uint64_t)(n - u - 2); /* candidates u+2 .. n-1 */
        uint64_t np = 0;
        /* Floyd: k distinct indices out of [0, cnt) */
        for (uint64_t j = cnt - k; j < cnt; j++) {
            uint32_t t = (uint32_t)sm64_range(&s, 0, j);
            uint32_t x = mark[t] == u + 1 ? (uint32_t)j : t;
            mark[x] = u + 1;
            pick[np++] = x;
        }
        qsort(pick, np, sizeof(uint32_t), cmp_u32);
        col[e] = u + 1;
        w[e] = 1;
        e++;
        for (uint64_t q = 0; q < np; q++) {
            uint32_t v = u + 2 + pick[q];
            col[e] = v;
            w[e] = 2u * (v - u);
            e++;
        }
    }
    row_ptr[n] = e;
    free(pick);
    free(mark);
    free(deg);
}

/* -------------------------------------------------- heap update batches */

/*
 * Closed-loop generator of parallel-bucket-heap update batches.  It keeps its
 * own record of which keys it believes are live and at which priority, from
 * the batches it issued and the extractions the caller reports back through
 * hs_observe_extracted().  It never decides by itself which keys leave; it
 * has no priority-queue logic.
 *
 * One batch of `batch` distinct keys: half are decreases of keys it records
 * as live (new priority uniform in [0, current)), the rest are keys it
 * records as not live, with priority uniform in [0, 2^32).  When fewer live
 * keys than half a batch exist, the batch is topped up with new keys.
 */
typedef struct {
    uint32_t key_space;
    uint64_t s;
    uint32_t *live;      /* dense list of live keys */
    int64_t *pos;        /* key -> index in live[], or -1 */
    uint32_t *prio;      /* key -> recorded priority (valid if live) */
    uint32_t *stamp;     /* key -> last batch that used it */
    uint32_t nlive;
    uint32_t round;
} gen_heap_stream;

void *hs_create(uint32_t key_space, uint64_t seed)
{
    gen_heap_stream *h = (gen_heap_stream *)calloc(1, sizeof(*h));
    h->key_space = key_space;
    h->s = stream_seed(seed, 5);
    h->live = (uint32_t *)malloc(sizeof(uint32_t) * key_space);
    h->pos = (int64_t *)malloc(sizeof(int64_t) * key_space);
    h->prio = (uint32_t *)malloc(sizeof(uint32_t) * key_space);
    h->stamp = (uint32_t *)calloc(key_space, sizeof(uint32_t));
    for (uint32_t k = 0; k < key_space; k++) h->pos[k] = -1;
    return h;
}

void hs_destroy(void *p)
{
    gen_heap_stream *h = (gen_heap_stream *)p;
    if (!h) return;
    free(h->live); free(h->pos); free(h->prio); free(h->stamp); free(h);
}

uint32_t hs_nlive(void *p) { return ((gen_heap_stream *)p)->nlive; }

static void hs_add_live(gen_heap_stream *h, uint32_t k, uint32_t prio)
{
    if (h->pos[k] < 0) {
        h->pos[k] = h->nlive;
        h->live[h->nlive++] = k;
    }
    h->prio[k] = prio;
}

static void hs_remove_live(gen_heap_stream *h, uint32_t k)
{
    int64_t p = h->pos[k];
    if (p < 0) return;
    uint32_t last = h->live[--h->nlive];
    h->live[p] = last;
    h->pos[last] = p;
    h->pos[k] = -1;
}

/* Returns the number of pairs written (== batch unless the key space runs out). */
uint32_t hs_next_batch(void *p, uint32_t batch, uint32_t *keys, uint32_t *prios)
{
    gen_heap_stream *h = (gen_heap_stream *)p;
    h->round++;
    uint32_t stamp = h->round;
    uint32_t out = 0;
    uint32_t want_dec = batch / 2;
    if (want_dec > h->nlive) want_dec = h->nlive;
    /* decreases of live keys */
    uint32_t tries = 0;
    while (out < want_dec && tries < 64u * batch) {
        tries++;
        uint32_t k = h->live[sm64_range(&h->s, 0, h->nlive - 1)];
        if (h->stamp[k] == stamp || h->prio[k] == 0) continue;
        uint32_t np = (uint32_t)sm64_range(&h->s, 0, (uint64_t)h->prio[k] - 1);
        h->stamp[k] = stamp;
        keys[out] = k;
        prios[out] = np;
        out++;
    }
    /* new keys (not live) */
    uint64_t free_keys = (uint64_t)h->key_space - h->nlive;
    tries = 0;
    uint32_t ndec = out;
    while (out < batch && free_keys > (uint64_t)(out - ndec) && tries < 1024u * batch) {
        tries++;
        uint32_t k = (uint32_t)sm64_range(&h->s, 0, h->key_space - 1);
        if (h->pos[k] >= 0 || h->stamp[k] == stamp) continue;
        h->stamp[k] = stamp;
        keys[out] = k;
        prios[out] = (uint32_t)sm64_next(&h->s);
        out++;
    }
    /* record: decreases keep min semantics, new keys become live */
    for (uint32_t i = 0; i < out; i++) hs_add_live(h, keys[i], prios[i]);
    return out;
}

void hs_observe_extracted(void *p, const uint32_t *keys, uint32_t count)
{
    gen_heap_stream *h = (gen_heap_stream *)p;
    for (uint32_t i = 0; i < count; i++)
        if (keys[i] < h->key_space) hs_remove_live(h, keys[i]);
}
