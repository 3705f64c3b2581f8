/*
 * pbh.h -- C ABI of the GB300 parallel bucket heap (parBucketHeap) and the
 * parallel Dijkstra (parDijkstra) it drives.
 *
 * Paper: K. Berney, J. Iacono, B. Karsin, N. Sitchinava, "A Parallel Priority
 * Queue with Fast Updates for GPU Architectures" (arXiv 1908.09378).
 *
 * Conventions for every call
 *   - Pointers named d_* are device pointers (caller-owned CUDA memory);
 *     pointers named h_* are host pointers.  Nothing is freed by the library
 *     except the opaque handle it allocated.
 *   - Calls taking a cudaStream_t are asynchronous on that stream unless
 *     marked "synchronises".  Errors found on the host (bad arguments) are
 *     returned at once; errors found on the device (a key out of range, a
 *     capacity overflow, an expired bounded wait) are latched in a status word
 *     inside the workspace and returned by the next synchronising call
 *     (pbh_size, pbh_sync, sssp_stats).
 *   - No call throws; no call aborts the process; no device code traps.
 *     Every device-side wait is bounded (one second by default) and reports
 *     PBH_E_TIMEOUT instead of hanging.
 *   - Element = (key, priority).  The heap orders elements by the packed
 *     64-bit word (priority << 32) | key, so ties in priority are broken by
 *     the smaller key.  This total order is the only order the library uses.
 */
#ifndef PBH_H
#define PBH_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PBH_OK = 0,
    PBH_E_INVAL = 1,    /* bad argument: null pointer, key >= key_space, count > d, r > d, source >= n, d < max degree */
    PBH_E_NOMEM = 2,    /* workspace smaller than *_workspace_bytes() */
    PBH_E_CAPACITY = 3, /* more live elements than the heap's capacity */
    PBH_E_RANGE = 4,    /* a tentative distance does not fit the packed word (see sssp_run) */
    PBH_E_TIMEOUT = 5,  /* a bounded device wait or a query's time limit expired */
    PBH_E_CUDA = 6      /* a CUDA runtime call failed; see pbh_last_error() */
} pbh_status;

/* ------------------------------------------------------------------ heap */

typedef struct pbh pbh_t; /* opaque, library-owned */

/*
 * Heap parameters (Section 2.2).
 *   key_space: keys are 0 .. key_space-1 (key_space <= 2^31).
 *   d:         the largest BulkUpdate and extract batch ("d" of Section 2.2).
 *              Bucket B_i holds d * 2^(2i+1) and signal buffer S_i holds
 *              d * 2^(2i) elements.
 *   capacity:  the most live elements at any time (the "n" of Section 2.2);
 *              0 means key_space.  The heap has q = ceil(log4(capacity/d)) + 1
 *              levels.
 */
typedef struct {
    uint32_t key_space;
    uint32_t d;
    uint64_t capacity;
} pbh_params;

/* Bytes of device workspace pbh_create needs for these parameters (0 if invalid). */
size_t pbh_workspace_bytes(const pbh_params *params);

/*
 * Create an empty heap in caller-owned device memory d_workspace (at least
 * pbh_workspace_bytes(params) bytes, 256-byte aligned).  The workspace must
 * stay allocated and untouched until pbh_destroy.  Initialisation is enqueued
 * on `stream`; all later calls must use the same stream (or order themselves
 * after it).  Section 2.2 (levels, capacities), Algorithm 1 (state).
 */
pbh_status pbh_create(pbh_t **out, const pbh_params *params, void *d_workspace, size_t ws_bytes,
                      cudaStream_t stream);

/*
 * BulkUpdate(U) of Section 1.2 / Section 2.2 for U = {(d_keys[i], d_prios[i])},
 * count <= d, device arrays.  Semantics: min-semantics decrease-or-insert.
 * A key that is not live is inserted; a live key takes the new priority only
 * if it is smaller (the paper assumes decreases, Section 1.2 footnote); several
 * pairs with one key keep the smallest priority.  Followed by Resolve(0) and
 * the resolution schedule of Theorem 3 (Resolve(i) after every fourth
 * Resolve(i-1)).  Keys >= key_space are ignored and latch PBH_E_INVAL.
 * count == 0 is a no-op.  Asynchronous.
 */
pbh_status pbh_bulk_update(pbh_t *h, const uint32_t *d_keys, const uint32_t *d_prios, uint32_t count);

/*
 * update(e) of Section 1.2 with the replace its footnote describes for
 * general (not only decreasing) updates: each pair (d_keys[i], d_prios[i]),
 * count <= d, device arrays, sets its key's priority, up or down, and a key
 * that is not live is inserted.  Pairs are timestamped by their position:
 * of several pairs with one key the last wins.  A pair equal to the live
 * element changes nothing.  The replaced copies become stale and every merge
 * that meets one drops it.  Followed by Resolve(0) and the schedule.  Keys
 * >= key_space are ignored and latch PBH_E_INVAL.  count == 0 is a no-op.
 * Asynchronous.
 */
pbh_status pbh_assign(pbh_t *h, const uint32_t *d_keys, const uint32_t *d_prios, uint32_t count);

/*
 * delete(e) of Section 1.2 for every key in d_keys[0, count), count <= d
 * (device array): a live key stops being live; keys that are not live, and
 * repeats, are ignored.  The paper moves a DEL element down the levels
 * (Section 2.2); here the key's live-word entry is cleared, which makes every
 * stored copy stale at once, and B_0 is filtered before the call returns on
 * the stream, so no later extract returns a deleted key.  Followed by
 * Resolve(0) and the schedule.  Keys >= key_space are ignored and latch
 * PBH_E_INVAL.  count == 0 is a no-op.  Asynchronous.
 */
pbh_status pbh_delete(pbh_t *h, const uint32_t *d_keys, uint32_t count);

/*
 * extractMin generalised to the r smallest (Section 1.2; r = 1 is the
 * paper's operation), r <= d.  Writes min(r, size) elements in ascending
 * (priority, key) order to d_keys_out[] / d_prios_out[] (device arrays of at
 * least r entries) and their number to *d_count_out (device), so the call can
 * be captured in a CUDA graph.  The extracted keys stop being live; updating
 * one later inserts it again.  Followed by Resolve(0) and the schedule.
 * r == 0 writes a count of 0.  Asynchronous.
 */
pbh_status pbh_extract_min(pbh_t *h, uint32_t r, uint32_t *d_keys_out, uint32_t *d_prios_out,
                           uint32_t *d_count_out);

/*
 * A sequence of heap operations in one launch, with the levels resolved
 * concurrently (Section 2.2.1, Figure 2, Theorem 3).  The CTAs of the launch
 * form two groups: the operation group runs the operations in order, every
 * Resolve(0) and every Resolve(1); the deep group (deep_ctas CTAs, at most
 * half the launch) runs every Resolve(2) and the deeper resolves it
 * triggers.  Resolve(2) number k starts once Resolve(1) number 4k has
 * finished and finishes before Resolve(1) number 4k+1 starts, so it overlaps
 * the operations in between, whose resolves touch levels 0 and 1 only.  Every
 * wait between the groups is bounded (PBH_E_TIMEOUT).  deep_ctas = 0 runs
 * the same schedule phase by phase on one group.  Results are the same as
 * calling pbh_bulk_update / pbh_extract_min for each operation in turn.
 *
 * ops: host array of nops operations (copied before the call returns; any
 * number, run in launches of 4096).  For PBH_OP_BULK_UPDATE: count <= d
 * pairs in d_keys / d_prios (device).  For PBH_OP_EXTRACT: r <= d; outputs as
 * pbh_extract_min (device arrays of at least r entries, count on the device).
 * The device arrays must stay valid until the work has run.  Asynchronous.
 */
#define PBH_OP_BULK_UPDATE 0u
#define PBH_OP_EXTRACT 1u
typedef struct {
    uint32_t kind;
    uint32_t count;
    uint32_t r;
    uint32_t reserved; /* 0 */
    const uint32_t *d_keys;
    const uint32_t *d_prios;
    uint32_t *d_keys_out;
    uint32_t *d_prios_out;
    uint32_t *d_count_out;
} pbh_op;
pbh_status pbh_run_ops(pbh_t *h, const pbh_op *ops, uint32_t nops, uint32_t deep_ctas);

/* Number of live elements.  Synchronises; returns any latched device error. */
pbh_status pbh_size(pbh_t *h, uint64_t *h_out);

/* Wait for the heap's stream; returns any latched device error. Synchronises. */
pbh_status pbh_sync(pbh_t *h);

/*
 * Debug check of the level invariants (Section 2.1: B_i <= B_j for j > i;
 * Algorithm 1: capacities, every run sorted, thresholds p_i separating the
 * levels; every live key stored).  Writes a bit mask of violated invariants
 * to *h_violations (0 = all hold) and the number of physically stored
 * elements to *h_stored.  A key that pbh_assign sets back to a word it held
 * before, while a stale copy of that word is still stored deeper, has two
 * valid copies of one word until a merge meets them; such a key is counted
 * once and its copies are not checked against the thresholds (extract stays
 * exact).  Synchronises.  Meant for tests.
 */
pbh_status pbh_validate(pbh_t *h, uint32_t *h_violations, uint64_t *h_stored);

/* Release the handle (not the workspace).  Synchronises. */
pbh_status pbh_destroy(pbh_t *h);

/* ----------------------------------------------------------------- SSSP */

/* CSR graph in device memory: arcs of vertex u are col[row_ptr[u] .. row_ptr[u+1]). */
typedef struct {
    uint32_t n;
    uint64_t m;
    const uint64_t *row_ptr; /* device, n + 1 entries */
    const uint32_t *col;     /* device, m entries */
} csr_t;

/*
 * Options of parDijkstra (Section 4.1).  Zero fields take defaults.
 *   r:     extract width: vertices taken from the heap per round (the paper
 *          uses 1).  The effective width is min(r, d / max_out_degree).
 *   d:     BulkUpdate batch size and heap parameter d (must be >= the
 *          largest out-degree; the paper sets d = maximum degree).
 *   cta:   team that runs the query: 0 = one cooperative grid over the
 *          whole GPU, 1 = one CTA, 2..16 = one thread-block cluster of that
 *          many CTAs (hardware cluster barrier), 17..4096 = one cooperative
 *          grid of exactly that many CTAs (PBH_E_INVAL if they cannot all
 *          be resident at once).
 *   flags: bits 0-3: CTAs per SM of the whole-GPU grid (0 = default);
 *          SSSP_SETTLE (bit 4): each round also extracts every vertex at the
 *          front of B_0 whose tentative distance is at most the heap minimum
 *          plus the smallest arc weight (such a vertex is final: any other
 *          path reaches it through a heap vertex and at least one more arc),
 *          up to d / max_out_degree vertices.  Distances are the same; the
 *          number of rounds falls, most when r is small (r = 1 is the
 *          paper's setting).  Costs one pass over the weights per query.
 *          SSSP_DEBUG_STALL (bit 8): for tests of the timeout path only.
 *          On the whole-GPU team, the first CTA withholds its arrival at the
 *          query's first device-wide barrier, so every CTA's bounded wait
 *          (wait_us) expires and the query ends with PBH_E_TIMEOUT; all
 *          work before that barrier is complete, so nothing reads unready
 *          data.  Ignored by the one-CTA and cluster teams.
 *          Other bits reserved, 0.
 *   limit_ms: bound on the query's device run time in milliseconds; past
 *          it the query stops at the end of a round with PBH_E_TIMEOUT.
 *          0 = 60 s + 0.1 ms per vertex (r = 1 needs one round per vertex).
 *   wait_us: bound on each device-wide barrier wait of the whole-GPU team
 *          in microseconds (PBH_E_TIMEOUT when it expires); 0 = 1 s.
 */
#define SSSP_SETTLE 0x10u
#define SSSP_DEBUG_STALL 0x100u
typedef struct {
    uint32_t r;
    uint32_t d;
    uint32_t cta;
    uint32_t flags;
    uint32_t limit_ms;
    uint32_t wait_us;
} sssp_opts;

/* Bytes of device workspace sssp_run needs for n vertices and these options. */
size_t sssp_workspace_bytes(uint32_t n, const sssp_opts *opts);

/*
 * opts == NULL lets the library choose: r = 512, d = 2^16, and the team by
 * size: one 16-CTA cluster for graphs of at most 2^19 arcs, else the whole
 * GPU (the fastest teams measured on GB300 for grids of 64x64 and 256x256 and
 * for banded graphs of 2^14 to 2^20 vertices).
 *
 * Single-source shortest paths by parDijkstra (Section 4.1): rounds of
 * extract-min of the r smallest tentative distances from a parallel bucket
 * heap, relaxation of all their out-arcs in parallel, and a BulkUpdate of the
 * improved (distance, vertex) pairs; until the heap is empty.  The whole loop
 * runs on the device in one launch (no host round trip per round).
 *
 * d_weights: device, m arc weights (uint32, >= 0).  d_dist_out: device,
 * n entries; receives the exact distance (uint64) of every vertex, and
 * UINT64_MAX for unreachable ones.  d_workspace: at least
 * sssp_workspace_bytes(n, opts) bytes.  During the run d_dist_out holds
 * packed (distance << k) | vertex words with k = ceil(log2 n); a tentative
 * distance above 2^(64-k) - 2 latches PBH_E_RANGE.  Asynchronous.
 */
pbh_status sssp_run(const csr_t *g, const uint32_t *d_weights, uint32_t source, uint64_t *d_dist_out,
                    const sssp_opts *opts, void *d_workspace, size_t ws_bytes, cudaStream_t stream);

/*
 * sssp_run from HOST buffers: copies the CSR arrays and weights (h_row_ptr,
 * h_col, h_weights; pinned memory gives full copy bandwidth) into device
 * workspace, runs, and copies the distances back to h_dist_out.  Needs
 * sssp_host_workspace_bytes(n, m, opts) bytes of device workspace.
 * Synchronises (the distances are on the host when it returns).
 */
size_t sssp_host_workspace_bytes(uint32_t n, uint64_t m, const sssp_opts *opts);
pbh_status sssp_run_host(uint32_t n, uint64_t m, const uint64_t *h_row_ptr, const uint32_t *h_col,
                         const uint32_t *h_weights, uint32_t source, uint64_t *h_dist_out,
                         const sssp_opts *opts, void *d_workspace, size_t ws_bytes, cudaStream_t stream);

/*
 * Allocation-free variant of sssp_run, for callers that cannot allocate
 * device memory when they run a query: a process under a fixed device-memory
 * budget, a custom allocator that must not grow, or a code path where a
 * cudaMalloc would stall the device.  The paper has no counterpart; this is
 * a library convenience.  Same arguments and results as sssp_run, except
 * that the workspace is a static scratch array of 32 MiB inside the library
 * (allocated on every device that loads the library, held until the process
 * exits) and nothing is allocated per call.  A query whose
 * sssp_workspace_bytes(n, opts) exceeds 32 MiB fails with PBH_E_NOMEM
 * (with the default options, n = 2^18 still fits and n = 2^19 does not).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.  Every call shares the one array and
 * finds the previous call's contents, which it overwrites; calls that
 * overlap on the GPU race on it, so serialise them (one stream, one host
 * thread at a time).  Synchronises: returns when the query has finished,
 * with its latched device status.
 */
pbh_status sssp_run_noalloc(const csr_t *g, const uint32_t *d_weights, uint32_t source, uint64_t *d_dist_out,
                            const sssp_opts *opts, cudaStream_t stream);

/* Counters of the last run in a workspace (synchronises; returns its latched error).
 * The same header counts a heap's operations: see pbh_stats. */
typedef struct {
    uint64_t rounds;          /* extract-relax-update rounds */
    uint64_t extracted;       /* vertices taken from the heap (>= reached vertices when r > 1) */
    uint64_t relaxations;     /* arcs scanned */
    uint64_t improvements;    /* arcs that lowered a tentative distance (BulkUpdate elements) */
    uint64_t stale_dropped;   /* superseded elements dropped while merging */
    uint64_t merged;          /* elements passed through level merges */
    uint64_t resolves[16];    /* Resolve(i) executions per level */
    uint64_t t_relax_ns;      /* device time per phase, seen by the first CTA (nanoseconds; heap
                                 operations only: queries compile the timers out, 0) */
    uint64_t t_sort_ns;       /*   sorting the BulkUpdate batch into S_0 */
    uint64_t t_empty0_ns;     /*   Empty(S_0) */
    uint64_t t_fill0_ns;      /*   Fill(B_0) */
    uint64_t t_deeper_ns;     /*   Resolve(i), i >= 1 */
    uint64_t t_ensure_ns;     /*   on-demand fill cascade before an extract */
    uint64_t barriers;        /* team barriers taken */
    uint32_t levels;          /* q */
    uint32_t r_eff;           /* extract width used */
    uint32_t max_degree;      /* largest out-degree seen */
    uint32_t status;          /* latched pbh_status */
    uint64_t settled;         /* vertices extracted beyond r by SSSP_SETTLE */
} sssp_stats_t;
pbh_status sssp_stats(const void *d_workspace, sssp_stats_t *h_out, cudaStream_t stream);

/* Counters of a heap since pbh_create, in the same record: merged (elements
 * passed through level merges, Algorithm 1), stale_dropped, resolves[i]
 * (Resolve(i) executions, Theorem 3), barriers and the phase times.  The
 * SSSP-only fields are 0.  Synchronises; returns any latched error. */
pbh_status pbh_stats(pbh_t *h, sssp_stats_t *h_out);

/* ------------------------------------------------------------- batched */

/* One query of a batch: its own graph, weights, source, output and team. */
typedef struct {
    csr_t g;
    const uint32_t *d_weights;
    uint32_t source;
    uint64_t *d_dist_out;
    uint32_t r;   /* 0 = default */
    uint32_t d;   /* 0 = default (>= max degree) */
    uint32_t cta; /* team: 0 or 1 = one CTA; 2..16 = one thread-block cluster of that many CTAs */
} sssp_query;

/*
 * Many independent queries in one persistent launch per team size: each CTA
 * (or, for queries with cta >= 2, each thread-block cluster) takes queries
 * from a device work queue (largest first, by the order the library sorts
 * them in) and runs each with its own heap, distances and counters.  The
 * cluster launches run on a library-owned second stream, forked from and
 * joined back to `stream`, beside the one-CTA launch; each gets a share of
 * the SMs in proportion to its share of the work (vertices + arcs).  Results
 * are identical to sssp_run on each query alone.  d_workspace must hold
 * sssp_batch_workspace_bytes(queries, nq) bytes.  `queries` is a host array.
 * Asynchronous.  Per-query status: sssp_batch_status.
 */
size_t sssp_batch_workspace_bytes(const sssp_query *queries, uint32_t nq);
pbh_status sssp_batch_run(const sssp_query *queries, uint32_t nq, void *d_workspace, size_t ws_bytes,
                          cudaStream_t stream);
/* Latched status of every query of the last batch in this workspace
 * (synchronises): low 16 bits = pbh_status, high 16 bits = the device site
 * that raised it (a diagnostic code, 0 when the status is PBH_OK). */
pbh_status sssp_batch_status(const void *d_workspace, uint32_t nq, uint32_t *h_status,
                             uint64_t *h_rounds, cudaStream_t stream);

/* -------------------------------------------------------------- serving */

/*
 * Continuous-batching SSSP server: ONE persistent launch whose CTAs take
 * queries from a request ring in pinned, device-mapped host memory (library
 * allocated) as soon as they are published, each query with its own heap and
 * distances in caller-provided device memory.  Queries published while
 * others run start as CTAs free up, so their work overlaps on the device.
 * Results are identical to sssp_run on each query alone.
 *
 * srv_create: `slots` ring entries; `ctas` resident CTAs (0 = every SM at
 * full occupancy); d_workspace of srv_workspace_bytes() bytes (claim
 * counter).  Launches the server on `stream`, which stays busy until
 * srv_stop.
 * srv_submit: publish one query; d_query_ws (256-byte aligned) of at least
 * srv_query_workspace_bytes(q) bytes holds its heap and counters (its status
 * and counters are read with sssp_stats(d_query_ws, ...) after completion).
 * *ticket receives the request number.  PBH_E_CAPACITY if the ring slot of
 * this ticket (ticket % slots) still holds an unfinished request.
 * srv_completion_arrays: host pointers to the per-slot completion words
 * (done[ticket % slots] == ticket + 1 once request `ticket` has finished;
 * its device globaltimer start/end in t_begin / t_end).
 * srv_stop: no more requests; idle CTAs leave; waits for the launch.  Every
 * wait is bounded: a CTA whose wait for a request sees the host silent (no
 * request, no srv_heartbeat) for longer than the idle limit (60 s unless
 * srv_idle_limit set another) leaves and latches PBH_E_TIMEOUT.
 */
typedef struct pbh_server pbh_server_t;
size_t srv_workspace_bytes(void);
size_t srv_query_workspace_bytes(const sssp_query *q);
pbh_status srv_create(pbh_server_t **out, uint32_t slots, uint32_t ctas, void *d_workspace, size_t ws_bytes,
                      cudaStream_t stream);
/* srv_create with a team per request: team = 1 is srv_create; team = 2..16
 * runs each request on one thread-block cluster of that many CTAs (for large
 * queries, whose one-CTA run would set the latency tail), with `ctas` CTAs
 * in all (a multiple of team; PBH_E_INVAL if not every cluster can be
 * resident at once).  Queries submitted to it have cta == team, and their
 * workspace is srv_query_workspace_bytes for that cta.  Two servers, one per
 * team, run side by side when their CTAs fit the GPU together. */
pbh_status srv_create_team(pbh_server_t **out, uint32_t slots, uint32_t ctas, uint32_t team, void *d_workspace,
                           size_t ws_bytes, cudaStream_t stream);
pbh_status srv_submit(pbh_server_t *s, const sssp_query *q, void *d_query_ws, size_t ws_bytes, uint64_t *ticket);
pbh_status srv_completion_arrays(pbh_server_t *s, uint64_t **done, uint64_t **t_begin, uint64_t **t_end,
                                 uint32_t *slots);
pbh_status srv_stop(pbh_server_t *s);
/* The first half of srv_stop: tells the server's CTAs to leave once idle,
 * without waiting.  With two servers side by side, request both stops before
 * waiting for either (srv_stop): a CTA of one launch may be scheduled only
 * when a CTA of the other leaves. */
pbh_status srv_request_stop(pbh_server_t *s);
/* A server CTA waiting for its next request gives up, and the server latches
 * PBH_E_TIMEOUT (reported by srv_stop), once the host has been silent for the
 * idle limit: no request published and no heartbeat.  srv_heartbeat tells
 * the waiting CTAs that the host is alive (call it while a stream is being
 * served); srv_idle_limit sets the limit in nanoseconds (0 restores the
 * default of 60 s) and applies to waits in progress too. */
pbh_status srv_heartbeat(pbh_server_t *s);
pbh_status srv_idle_limit(pbh_server_t *s, uint64_t ns);
pbh_status srv_destroy(pbh_server_t *s);

/* --------------------------------------------------------------- misc */

/* Thread-local text of the last error. */
const char *pbh_last_error(void);

/* Library version string. */
const char *pbh_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PBH_H */
