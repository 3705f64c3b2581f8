/*
 * oracle.c -- plain, slow, obviously correct CPU reference for the parity
 * tests of the parallel bucket heap and of parallel Dijkstra.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this code.  It shares nothing with the CUDA
 * library: no headers, no helpers, no constants.
 *
 * Contents
 *   oracle_dijkstra      sequential Dijkstra over a binary heap with lazy
 *                        deletion (Section 1: classical SSSP; the problem of
 *                        Section 1.1 and the per-round semantics of Section 4.1)
 *   oracle_dijkstra_counts  the same run's counters: settled vertices,
 *                        scanned arcs, successful relaxations
 *   oracle_bellman_ford  the plain O(nm) relaxation sweep (Section 1), used to
 *                        pin Dijkstra on tiny graphs
 *   oracle_check_sssp    the optimality certificate of a distance vector
 *   oracle_hop_depth     minimum hop count of a shortest path, maximised
 *   oracle_reached_edges sum of out-degrees of reached vertices (GTEPS numerator)
 *   opq_*                a sorted-array priority queue with the ADT of
 *                        Section 1.2 (extractMin, update, BulkUpdate, delete;
 *                        update both with the decrease-only assumption of the
 *                        paper and with the footnote's timestamped replace)
 *
 * Distances are uint64; "unreachable" is UINT64_MAX.  The paper starts every
 * tentative distance at "-infinity" in Section 1; shortest paths are a
 * minimisation, so this reads it as +infinity.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define INF64 UINT64_MAX

/* ------------------------------------------------------ binary min-heap */

typedef struct {
    uint64_t d;
    uint32_t v;
} hent;

static int hless(hent a, hent b)
{
    return a.d < b.d || (a.d == b.d && a.v < b.v);
}

static void hpush(hent *h, uint64_t *len, hent x)
{
    uint64_t i = (*len)++;
    h[i] = x;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (!hless(h[i], h[p])) break;
        hent t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

static hent hpop(hent *h, uint64_t *len)
{
    hent top = h[0];
    h[0] = h[--(*len)];
    uint64_t i = 0, n = *len;
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < n && hless(h[l], h[s])) s = l;
        if (r < n && hless(h[r], h[s])) s = r;
        if (s == i) break;
        hent t = h[i]; h[i] = h[s]; h[s] = t;
        i = s;
    }
    return top;
}

/*
 * Dijkstra: repeatedly take the unvisited vertex of minimum tentative
 * distance and relax all its out-arcs.  Stale heap entries (a vertex pushed
 * again with a smaller distance) are skipped when popped.
 * parent (nullable) receives the tree parent of each reached vertex
 * (UINT32_MAX for the source and for unreached vertices).
 * counts (nullable) receives [0] vertices settled, [1] arcs scanned, [2]
 * successful relaxations: arcs whose new distance was strictly below the
 * tentative one (each becomes one heap element; parDijkstra with r = 1,
 * Section 4.1, stages the same improvements).
 * Returns the number of vertices settled.
 */
static uint64_t dijkstra_run(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, const uint32_t *w,
                             uint32_t source, uint64_t *dist, uint32_t *parent, uint64_t *counts)
{
    for (uint32_t v = 0; v < n; v++) {
        dist[v] = INF64;
        if (parent) parent[v] = UINT32_MAX;
    }
    if (source >= n) return 0;
    uint64_t m = row_ptr[n];
    hent *heap = (hent *)malloc(sizeof(hent) * (m + 2));
    unsigned char *done = (unsigned char *)calloc(n, 1);
    uint64_t len = 0, settled = 0, scanned = 0, improved = 0;
    dist[source] = 0;
    hpush(heap, &len, (hent){0, source});
    while (len > 0) {
        hent x = hpop(heap, &len);
        if (done[x.v] || x.d != dist[x.v]) continue;
        done[x.v] = 1;
        settled++;
        for (uint64_t e = row_ptr[x.v]; e < row_ptr[x.v + 1]; e++) {
            uint32_t v = col[e];
            uint64_t nd = x.d + w[e];
            scanned++;
            if (nd < dist[v]) {
                dist[v] = nd;
                improved++;
                if (parent) parent[v] = x.v;
                hpush(heap, &len, (hent){nd, v});
            }
        }
    }
    free(heap);
    free(done);
    if (counts) {
        counts[0] = settled;
        counts[1] = scanned;
        counts[2] = improved;
    }
    return settled;
}

uint64_t oracle_dijkstra(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, const uint32_t *w,
                         uint32_t source, uint64_t *dist, uint32_t *parent)
{
    return dijkstra_run(n, row_ptr, col, w, source, dist, parent, NULL);
}

/*
 * The counters of the same Dijkstra run (see dijkstra_run): counts[0..2] =
 * settled vertices, scanned arcs, successful relaxations.  The successful
 * relaxations U fix the heap traffic of the benchmark's roofline: each is one
 * heap word written once and read once.
 */
uint64_t oracle_dijkstra_counts(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, const uint32_t *w,
                                uint32_t source, uint64_t *dist, uint64_t *counts)
{
    return dijkstra_run(n, row_ptr, col, w, source, dist, NULL, counts);
}

/*
 * Bellman-Ford: relax every arc until a full sweep changes nothing (at most
 * n - 1 useful sweeps for non-negative weights).  Returns the sweeps made.
 */
uint64_t oracle_bellman_ford(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, const uint32_t *w,
                             uint32_t source, uint64_t *dist)
{
    for (uint32_t v = 0; v < n; v++) dist[v] = INF64;
    if (source >= n) return 0;
    dist[source] = 0;
    uint64_t sweeps = 0;
    for (uint32_t it = 0; it < n; it++) {
        int changed = 0;
        sweeps++;
        for (uint32_t u = 0; u < n; u++) {
            if (dist[u] == INF64) continue;
            for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
                uint64_t nd = dist[u] + w[e];
                if (nd < dist[col[e]]) {
                    dist[col[e]] = nd;
                    changed = 1;
                }
            }
        }
        if (!changed) break;
    }
    return sweeps;
}

/* Vertices reachable from source by arcs (BFS); out[v] = 1 if reachable. */
static void reach(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, uint32_t source,
                  unsigned char *out)
{
    memset(out, 0, n);
    if (source >= n) return;
    uint32_t *q = (uint32_t *)malloc(sizeof(uint32_t) * n);
    uint32_t qh = 0, qt = 0;
    out[source] = 1;
    q[qt++] = source;
    while (qh < qt) {
        uint32_t u = q[qh++];
        for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; e++)
            if (!out[col[e]]) {
                out[col[e]] = 1;
                q[qt++] = col[e];
            }
    }
    free(q);
}

/*
 * Optimality certificate of a distance vector dist for source s:
 *   counts[0]: dist[s] != 0
 *   counts[1]: arcs (u,v) with dist[u] finite and dist[u] + w < dist[v]
 *   counts[2]: reached v != s with no tight in-arc (dist[u] + w == dist[v])
 *   counts[3]: v whose finiteness disagrees with BFS reachability
 * Returns the total.  A vector passing all four is the exact distance vector.
 */
uint64_t oracle_check_sssp(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, const uint32_t *w,
                           uint32_t source, const uint64_t *dist, uint64_t *counts)
{
    uint64_t c[4] = {0, 0, 0, 0};
    if (source < n && dist[source] != 0) c[0]++;
    unsigned char *tight = (unsigned char *)calloc(n ? n : 1, 1);
    for (uint32_t u = 0; u < n; u++) {
        if (dist[u] == INF64) continue;
        for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
            uint32_t v = col[e];
            uint64_t nd = dist[u] + w[e];
            if (nd < dist[v]) c[1]++;
            if (nd == dist[v]) tight[v] = 1;
        }
    }
    unsigned char *r = (unsigned char *)malloc(n ? n : 1);
    reach(n, row_ptr, col, source, r);
    for (uint32_t v = 0; v < n; v++) {
        if (v != source && dist[v] != INF64 && !tight[v]) c[2]++;
        if ((dist[v] != INF64) != (r[v] != 0)) c[3]++;
    }
    free(r);
    free(tight);
    if (counts) memcpy(counts, c, sizeof(c));
    return c[0] + c[1] + c[2] + c[3];
}

/*
 * Hop depth H: for every reached vertex the fewest arcs on any shortest path
 * from the source (a BFS over tight arcs), maximised over vertices.  A
 * round-synchronous method needs at least H rounds to finish.
 * hops (nullable) receives the per-vertex value (UINT32_MAX if unreached).
 */
uint32_t oracle_hop_depth(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, const uint32_t *w,
                          uint32_t source, const uint64_t *dist, uint32_t *hops)
{
    uint32_t *h = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    for (uint32_t v = 0; v < n; v++) h[v] = UINT32_MAX;
    if (source >= n) {
        if (hops) memcpy(hops, h, sizeof(uint32_t) * n);
        free(h);
        return 0;
    }
    uint32_t *q = (uint32_t *)malloc(sizeof(uint32_t) * n);
    uint32_t qh = 0, qt = 0, H = 0;
    h[source] = 0;
    q[qt++] = source;
    while (qh < qt) {
        uint32_t u = q[qh++];
        if (h[u] > H) H = h[u];
        for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {
            uint32_t v = col[e];
            if (h[v] == UINT32_MAX && dist[u] != INF64 && dist[u] + w[e] == dist[v]) {
                h[v] = h[u] + 1;
                q[qt++] = v;
            }
        }
    }
    if (hops) memcpy(hops, h, sizeof(uint32_t) * n);
    free(q);
    free(h);
    return H;
}

/* Sum of out-degrees of the vertices with a finite distance. */
uint64_t oracle_reached_edges(uint32_t n, const uint64_t *row_ptr, const uint64_t *dist)
{
    uint64_t s = 0;
    for (uint32_t v = 0; v < n; v++)
        if (dist[v] != INF64) s += row_ptr[v + 1] - row_ptr[v];
    return s;
}

/* ------------------------------------------------ sorted-array priority queue */

/*
 * The priority-queue ADT of Section 1.2 over elements (value = key, priority):
 *   update(key, prio): insert, or replace a live element of the same key.
 *     Updates are decreases in the paper (footnote to Section 1.2); an update
 *     that does not lower a live key's priority leaves it unchanged, and
 *     several updates of one key in a batch keep the smallest priority.
 *     Updating a key that is not live (never inserted, or extracted) inserts it.
 *   BulkUpdate(U): update for every element of U.
 *   extractMin(r): remove and return the min(r, size) smallest elements in
 *     ascending (priority, key) order; r = 1 is the paper's extractMin.
 *
 * Storage: a sorted array of live elements packed as (prio << 32) | key, read
 * from a head offset, and a dense key -> priority table.
 */
typedef struct {
    uint32_t key_space;
    uint64_t *cur;   /* key -> live priority, or INF64 if not live */
    uint64_t *arr;   /* sorted live elements */
    uint64_t head, len, cap;
    uint64_t *tmp;
    uint64_t *batch; /* key -> best priority within the current batch */
} opq;

void *opq_create(uint32_t key_space)
{
    opq *q = (opq *)calloc(1, sizeof(opq));
    q->key_space = key_space;
    q->cur = (uint64_t *)malloc(sizeof(uint64_t) * (key_space ? key_space : 1));
    q->batch = (uint64_t *)malloc(sizeof(uint64_t) * (key_space ? key_space : 1));
    for (uint32_t k = 0; k < key_space; k++) q->cur[k] = q->batch[k] = INF64;
    q->cap = 1024;
    q->arr = (uint64_t *)malloc(sizeof(uint64_t) * q->cap);
    q->tmp = (uint64_t *)malloc(sizeof(uint64_t) * q->cap);
    return q;
}

void opq_destroy(void *p)
{
    opq *q = (opq *)p;
    if (!q) return;
    free(q->cur); free(q->batch); free(q->arr); free(q->tmp); free(q);
}

uint64_t opq_size(void *p) { return ((opq *)p)->len; }

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Returns the number of elements whose priority changed or that were inserted. */
uint64_t opq_bulk_update(void *p, const uint32_t *keys, const uint32_t *prios, uint32_t count)
{
    opq *q = (opq *)p;
    uint32_t *touched = (uint32_t *)malloc(sizeof(uint32_t) * (count ? count : 1));
    uint32_t nt = 0;
    /* 1. best priority per key within the batch, if it improves the live one */
    for (uint32_t i = 0; i < count; i++) {
        uint32_t k = keys[i];
        uint64_t pr = prios[i];
        if (k >= q->key_space) continue;
        if (q->cur[k] != INF64 && q->cur[k] <= pr) continue;
        if (q->batch[k] == INF64) touched[nt++] = k;
        if (pr < q->batch[k]) q->batch[k] = pr;
    }
    /* 2. new packed elements; the changed keys' old elements become stale */
    uint64_t *fresh = (uint64_t *)malloc(sizeof(uint64_t) * (nt ? nt : 1));
    for (uint32_t i = 0; i < nt; i++) {
        uint32_t k = touched[i];
        q->cur[k] = q->batch[k];
        q->batch[k] = INF64;
        fresh[i] = (q->cur[k] << 32) | k;
    }
    qsort(fresh, nt, sizeof(uint64_t), cmp_u64);
    /* 3. one linear merge of the surviving old elements with the fresh ones */
    uint64_t need = q->len + nt;
    if (need > q->cap) {
        while (q->cap < need) q->cap *= 2;
        q->tmp = (uint64_t *)realloc(q->tmp, sizeof(uint64_t) * q->cap);
    }
    uint64_t i = q->head, end = q->head + q->len, j = 0, o = 0;
    while (i < end || j < nt) {
        if (i < end) {
            uint64_t e = q->arr[i];
            if ((e >> 32) != q->cur[e & 0xFFFFFFFFu]) { i++; continue; } /* stale */
            if (j >= nt || e < fresh[j]) { q->tmp[o++] = e; i++; continue; }
        }
        q->tmp[o++] = fresh[j++];
    }
    if (q->cap > 0) {
        uint64_t *t = q->arr;
        q->arr = q->tmp;
        q->tmp = (uint64_t *)realloc(t, sizeof(uint64_t) * q->cap);
    }
    q->head = 0;
    q->len = o;
    free(fresh);
    free(touched);
    return nt;
}

uint32_t opq_extract_min(void *p, uint32_t r, uint32_t *keys_out, uint32_t *prios_out)
{
    opq *q = (opq *)p;
    uint64_t c = r < q->len ? r : q->len;
    for (uint64_t i = 0; i < c; i++) {
        uint64_t e = q->arr[q->head + i];
        uint32_t k = (uint32_t)(e & 0xFFFFFFFFu);
        if (keys_out) keys_out[i] = k;
        if (prios_out) prios_out[i] = (uint32_t)(e >> 32);
        q->cur[k] = INF64;
    }
    q->head += c;
    q->len -= c;
    return (uint32_t)c;
}

/* Drop the array elements that are no longer their key's live element. */
static void opq_compact(opq *q)
{
    uint64_t o = 0;
    for (uint64_t i = q->head; i < q->head + q->len; i++) {
        uint64_t e = q->arr[i];
        if ((e >> 32) == q->cur[e & 0xFFFFFFFFu]) q->arr[o++] = e;
    }
    q->head = 0;
    q->len = o;
}

/*
 * update(e) with the footnote of Section 1.2: e replaces the element of the
 * same key whatever the two priorities (a later timestamp wins).  Within one
 * batch the later position is the later timestamp, so the last element of
 * each key decides.  A key that is not live is inserted.  Returns the number
 * of keys whose live priority changed or that became live.
 */
uint64_t opq_assign(void *p, const uint32_t *keys, const uint32_t *prios, uint32_t count)
{
    opq *q = (opq *)p;
    uint32_t *touched = (uint32_t *)malloc(sizeof(uint32_t) * (count ? count : 1));
    uint32_t nt = 0;
    for (uint32_t i = 0; i < count; i++) { /* the last element of each key wins */
        uint32_t k = keys[i];
        if (k >= q->key_space) continue;
        if (q->batch[k] == INF64) touched[nt++] = k;
        q->batch[k] = prios[i];
    }
    uint64_t changed = 0;
    for (uint32_t i = 0; i < nt; i++) {
        uint32_t k = touched[i];
        if (q->cur[k] != q->batch[k]) {
            q->cur[k] = q->batch[k];
            touched[changed++] = k;
        }
        q->batch[k] = INF64;
    }
    opq_compact(q); /* replaced elements leave */
    uint64_t need = q->len + changed;
    if (need > q->cap) {
        while (q->cap < need) q->cap *= 2;
        q->arr = (uint64_t *)realloc(q->arr, sizeof(uint64_t) * q->cap);
        q->tmp = (uint64_t *)realloc(q->tmp, sizeof(uint64_t) * q->cap);
    }
    for (uint64_t i = 0; i < changed; i++) q->arr[q->len + i] = (q->cur[touched[i]] << 32) | touched[i];
    q->len += changed;
    qsort(q->arr, q->len, sizeof(uint64_t), cmp_u64);
    free(touched);
    return changed;
}

/* delete(e) of Section 1.2: the key stops being live.  Keys that are not
 * live are ignored.  Returns the number of keys removed. */
uint64_t opq_delete(void *p, const uint32_t *keys, uint32_t count)
{
    opq *q = (opq *)p;
    uint64_t gone = 0;
    for (uint32_t i = 0; i < count; i++) {
        uint32_t k = keys[i];
        if (k < q->key_space && q->cur[k] != INF64) {
            q->cur[k] = INF64;
            gone++;
        }
    }
    opq_compact(q);
    return gone;
}

/* Live priority of key (UINT64_MAX if not live). */
uint64_t opq_priority(void *p, uint32_t key)
{
    opq *q = (opq *)p;
    return key < q->key_space ? q->cur[key] : INF64;
}
