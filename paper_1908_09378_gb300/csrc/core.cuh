// core.cuh -- device side of the GB300 parallel bucket heap and parDijkstra.
//
// Structure
//   * Teams.  Every algorithm below is written once against a "team" of
//     CTAs: GridTeam = all CTAs of one cooperative launch (the whole GPU,
//     joined by a bounded grid barrier), CtaTeam = one CTA (joined by
//     __syncthreads).  The single-query path uses GridTeam; the batched path
//     runs one query per CtaTeam.
//   * Replicated control.  The heap's control state (level runs, thresholds,
//     schedule counters) lives in shared memory of every CTA.  All CTAs run
//     the same control code on the same values, so they take the same branch
//     without a leader broadcast; values produced by data-parallel phases
//     (e.g. how many elements survived a merge) are read back from global
//     memory after the team barrier.
//   * Data-parallel phases are merge-path merges (Green, McColl, Bader 2012)
//     over 2048-element tiles staged in shared memory, a validity filter, and
//     compaction.  All element runs are sorted by the packed 64-bit word.
//
// Paper: Berney, Iacono, Karsin, Sitchinava, "A Parallel Priority Queue with
// Fast Updates for GPU Architectures".  Section 2.2 (levels and capacities),
// Algorithm 1 (Resolve), Theorem 3 (schedule), Section 4.1 (parDijkstra).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pbhk {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr u64 INF = ~0ull;
constexpr int NT = 256;              // threads per CTA
constexpr int IPT = 8;               // items per thread in a tile (must be 8: one flag byte per thread)
constexpr int TILE = NT * IPT;       // elements per merge tile
constexpr int NWARPS = NT / 32;
constexpr int MAXQ = 16;             // most levels a heap may have
constexpr int FMAX = 1024;           // frontier vertices one CTA stages at a time
#if defined(PBH_BULK_TILES) && defined(PBH_BULK_RELAX)
#error "PBH_BULK_TILES and PBH_BULK_RELAX share the late flag: build one at a time"
#endif
constexpr u64 SPIN_NS = 1000000000ull; // default bound on every device-side wait (1 s)
constexpr u64 QUERY_NS = 60000000000ull; // default bound on one query's run time: 60 s ...
constexpr u64 QUERY_NS_PER_VERTEX = 100000ull; // ... plus 100 us per vertex (r = 1 takes one round per vertex)

// status codes (same values as pbh_status in include/pbh.h)
enum : u32 { ST_OK = 0, ST_INVAL = 1, ST_NOMEM = 2, ST_CAPACITY = 3, ST_RANGE = 4, ST_TIMEOUT = 5 };

// counters kept per heap / query
enum {
    STAT_ROUNDS = 0, STAT_EXTRACTED, STAT_RELAX, STAT_IMPROVE, STAT_STALE, STAT_MERGED,
    STAT_MAXDEG, STAT_REFF, STAT_LEVELS, STAT_RES0,
    // device time per phase (ns, seen by CTA 0) and team barriers taken
    STAT_T_RELAX = STAT_RES0 + MAXQ, STAT_T_SORT, STAT_T_EMPTY, STAT_T_FILL, STAT_T_DEEP, STAT_T_ENSURE,
    STAT_SYNCS, STAT_SETTLED, STAT_WMIN, STAT_N,
    // per-step tracing of a round (builds with PBH_PROBES only): SM cycles of
    // CTA 0 between consecutive probe points, summed over rounds
    STAT_PROBE0 = STAT_N, STAT_NPROBES = 24
};

// ------------------------------------------------------------ heap state

// One level i of the heap (Section 2.2): bucket B_i and signal buffer S_i,
// each a sorted run inside one of two ping-pong buffers, and threshold T_i
// (the paper's p_i): every element of B_i is <= T_i and every element stored
// at a deeper level is > T_i.  T_i = INF means "no bound" (the paper's p_l of
// the last level).
struct Level {
    u64 *B[2];
    u64 *S[2];
    u64 bufB, bufS;  // buffer sizes (elements)
    u64 capB, capS;  // d * 2^(2i+1), d * 2^(2i)
    u64 bhead, blen; // B_i = B[bsel][bhead, bhead + blen)
    u64 shead, slen; // S_i = S[ssel][shead, shead + slen)
    u64 T;
    u64 nres;        // Resolve(i) executions (Theorem 3 schedule)
    u32 bsel, ssel;
};

struct HeapState {
    u32 q;                // number of levels
    u32 reset_on_extract; // 1: extracted keys become not live (pbh API); 0: SSSP (distances only fall)
    u64 d;
    u64 keymask;          // key = word & keymask
    u64 key_space;
    u64 *cur;             // key -> the live packed word (INF if none): validity of stored elements
    u64 *U[2];            // BulkUpdate staging (d elements each); level 0's S buffers alias these
    u64 live;             // live elements (pbh API)
    u32 *mark;            // SSSP: key -> tag of the last round that staged it (one staged word per key and round)
    u32 settle;           // SSSP: also extract the vertices the settle criterion proves final
    Level L[MAXQ];
};

// Heap operations of the pbh API.
enum : int { OP_BULK = 0, OP_EXTRACT = 1, OP_DELETE = 2, OP_ASSIGN = 3 };

struct HeapCounters { // monotone counters of the pbh API, in the workspace header
    u64 inserted;      // keys that became live
    u64 extracted;     // elements returned by extract
    u64 deleted;       // live keys removed by delete
};

// Per-team global scratch.
struct Scratch {
    u64 *bar;           // grid barrier arrival counter (monotone)
    u32 *err;           // latched status word
    u64 *partials;      // per-CTA counts
    u64 *res;           // results of the last merge [0]=kept [1]=a_end [2]=last [3]=has_last
    unsigned char *bits;// validity flags of multi-tile merges (one byte per thread chunk)
    u64 *splits;        // merge-path starts of multi-tile merges
    u64 *ucount;        // number of staged BulkUpdate elements
    u64 *stats;         // STAT_N counters
    u64 wait_ns;        // bound on one barrier wait (0 = SPIN_NS)
    u32 stall;          // test only: CTA 0 withholds its first grid-barrier arrival
    u32 pad;
};

// Shared memory of one CTA.
struct Smem {
    HeapState hs;
    alignas(16) u64 win[TILE + 8]; // merge / sort window (16-byte aligned: bulk-copy destination)
    u64 keep[TILE + 8];  // compaction staging (also aliased by the relax arrays)
    u64 last[NT];        // last item of every thread (dedup predecessor)
    u64 bc[16];          // broadcast slots
    u64 mbar;            // mbarrier of the bulk copies (cp.async.bulk) into shared memory
    u64 tile_mbar;       // mbarrier of the merge tiles' bulk copies (PBH_BULK_TILES builds)
    u32 mbar_phase;      // its current phase parity
    u32 mbar_late;       // a wait on it expired in this phase
    u32 scan[NWARPS + 2];
    u64 scan64[NWARPS + 1];
};

static_assert(IPT == 8, "one flag byte per thread");
static_assert(3 * FMAX * 8 <= (2 * (TILE + 8)) * 8, "relax arrays must fit in win+keep");

// ----------------------------------------------------------- low level

__device__ __forceinline__ u64 ldg_cg(const u64 *p) { return __ldcg(p); }

__device__ __forceinline__ u64 ld_acquire(const u64 *p)
{
    u64 v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ u64 gtimer()
{
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Latch the first error: err[0] = status code, err[1] = the site that raised it.
// Per-CTA error state (shared memory): the status word of the query this CTA
// is running, for checks deep inside primitives that do not carry the team;
// a flag that this CTA raised or observed an error; and, under a grid team,
// the barrier counter, whose top bit an error sets so that every CTA learns
// of it at its next barrier and no barrier waits once one is set.
__shared__ u32 *s_err_sink;
__shared__ u64 *s_bar_sink;
__shared__ u32 s_err_flag;

constexpr u64 BAR_ERR = 1ull << 63;

// Thread 0, before the CTA's next __syncthreads.
__device__ __forceinline__ void g_err_sink_set(u32 *e, u64 *bar = nullptr)
{
    s_err_sink = e;
    s_bar_sink = bar;
    s_err_flag = 0;
}

// Latch (code, site) into the status word (the first error wins), flag the
// CTA and release the grid team's barriers.
__device__ __forceinline__ void raise_err(u32 *err, u32 code, u32 site)
{
    if (atomicCAS(err, 0u, code) == 0u) err[1] = site;
    s_err_flag = 1;
    if (s_bar_sink) atomicOr(s_bar_sink, BAR_ERR);
}
__device__ __forceinline__ u32 read_err(const u32 *err) { return *(volatile const u32 *)err; }

// Grid-barrier arrival: add 1 to the counter with release semantics.
__device__ __forceinline__ void bar_arrive(u64 *p)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(1ull) : "memory");
}

// Counter update that does not wait for the memory system (a reduction, not
// a load and a store): statistics stay off the critical path of a round.
__device__ __forceinline__ void stat_add(u64 *p, u64 v)
{
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Tracing hook: PBH_PROBE(team, k) adds the SM cycles CTA 0's thread 0 spent
// since its previous probe to stats[STAT_PROBE0 + k].  It compiles to nothing
// unless the library is built with -DPBH_PROBES (a tracing build).
#ifdef PBH_PROBES
__shared__ long long s_probe_t;
#define PBH_PROBE(t, k)                                                                 \
    do {                                                                                \
        if ((t).cta() == 0 && threadIdx.x == 0) {                                       \
            const long long now_ = clock64();                                          \
            stat_add((t).sc.stats + STAT_PROBE0 + (k), (u64)(now_ - s_probe_t));        \
            s_probe_t = now_;                                                           \
        }                                                                               \
    } while (0)
#define PBH_PROBE_START(t)                                    \
    do {                                                      \
        if ((t).cta() == 0 && threadIdx.x == 0) s_probe_t = clock64(); \
    } while (0)
// Per-CTA phase spans: PBH_SPAN_BEGIN marks the start in every CTA;
// PBH_SPAN_END(t, k) adds the CTA's cycles since then to slot k (a sum over
// CTAs) and raises slot k + 1 to the largest of them.
__shared__ long long s_span_t;
#define PBH_SPAN_BEGIN()                                \
    do {                                                \
        if (threadIdx.x == 0) s_span_t = clock64();     \
    } while (0)
#define PBH_SPAN_END(t, k)                                                              \
    do {                                                                                \
        if (threadIdx.x == 0) {                                                         \
            const u64 d_ = (u64)(clock64() - s_span_t);                                 \
            stat_add((t).sc.stats + STAT_PROBE0 + (k), d_);                             \
            atomicMax((t).sc.stats + STAT_PROBE0 + (k) + 1, d_);                        \
        }                                                                               \
    } while (0)
#else
#define PBH_PROBE(t, k) \
    do {                \
    } while (0)
#define PBH_PROBE_START(t) \
    do {                   \
    } while (0)
#define PBH_SPAN_BEGIN() \
    do {                 \
    } while (0)
#define PBH_SPAN_END(t, k) \
    do {                   \
    } while (0)
#endif

// --------------------------------------------------- bulk copies (TMA)
//
// 1-D bulk copies global -> shared memory (cp.async.bulk) completed on an
// mbarrier: one thread issues a copy of a whole contiguous segment; the
// barrier's transaction count tracks the bytes in flight.  Both addresses
// and the size must be multiples of 16 bytes.

__device__ __forceinline__ u32 smem_u32(const void *p)
{
    return (u32)__cvta_generic_to_shared(p);
}

// Thread 0, once per kernel, followed by a __syncthreads.
__device__ __forceinline__ void mbar_init(u64 *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The single arrival of a phase, announcing `bytes` of copies.
__device__ __forceinline__ void mbar_arrive_expect(u64 *bar, u32 bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, u32 bytes, u64 *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(u64 *bar, u32 parity)
{
    u32 ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait for the phase of `parity` to complete; false on expiry.
__device__ __forceinline__ bool mbar_wait(u64 *bar, u32 parity)
{
    u64 t0 = 0;
    for (u32 spins = 0; !mbar_test(bar, parity); spins++) {
        if ((spins & 63) == 0) {
            const u64 now = gtimer();
            if (t0 == 0)
                t0 = now;
            else if (now - t0 > SPIN_NS)
                return false;
        }
    }
    return true;
}

// Invalidate a barrier whose phase completed (before it is initialised again).
__device__ __forceinline__ void mbar_inval(u64 *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Order this thread's earlier generic-proxy view of global memory (what an
// acquire made visible) before its later bulk copies (the async proxy).
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// ------------------------------------------------------------------ teams

// Timed: the team records the device time per phase (STAT_T_*, CTA 0).
// Heap operations keep the timers; the SSSP query teams compile them out:
// the global-timer reads, even when skipped at run time, cost about 0.5 us
// per round of the whole-GPU query (they constrain the instruction schedule
// around the barriers).
template <bool Timed>
struct GridTeamT {
    static constexpr bool kSingle = false;
    static constexpr bool kTimed = Timed;
    static constexpr bool kSoftBarrier = true; // a software barrier with a bounded wait
    // Has an error been raised?  The CTA's own errors show at once, every
    // other CTA's from its next barrier on (the counter's top bit); a CTA
    // that acts on one earlier than another cannot hang it, since no barrier
    // waits once the bit is set.  Uniform within the CTA after a __syncthreads.
    __device__ __forceinline__ bool failed() const { return s_err_flag != 0; }
    Scratch sc;
    u64 gen = 0;   // barriers this CTA has completed (thread 0's copy is the one used)
    u64 nsync = 0;
    bool withhold = false; // skip the arrival of the next barrier (the stall test)
    __device__ __forceinline__ u32 ncta() const { return gridDim.x; }
    __device__ __forceinline__ u32 cta() const { return blockIdx.x; }
    // Call once at kernel start, before the first sync: the arrival counter
    // is a multiple of the grid size between launches, and this launch's
    // first barrier cannot complete before this CTA arrives.
    __device__ void init()
    {
        if (threadIdx.x == 0) gen = ld_acquire(sc.bar) / gridDim.x;
    }
    // Grid barrier: one arrival per CTA on a monotone counter, then wait
    // until the counter reaches the end of this barrier's generation.  The
    // wait is bounded; on expiry the status word latches ST_TIMEOUT and the
    // CTA continues, so the kernel winds down instead of hanging.
    __device__ void sync() { soft_barrier(sc, gridDim.x, gen, nsync, withhold); }

    // The barrier of a team of `size` CTAs on the counter sc.bar (shared by
    // GridTeam and the CTA groups of concurrent resolution).
    static __device__ void soft_barrier(const Scratch &sc, u32 size, u64 &gen, u64 &nsync, bool &withhold)
    {
        __syncthreads();
        if (threadIdx.x == 0) {
            // release arrival, acquire wait: the release is cumulative over
            // the CTA's writes that the __syncthreads above ordered before it,
            // and the acquire that sees the last arrival orders every CTA's
            // writes before this CTA's later reads (the __syncthreads below
            // extends that to its other threads).  Measured 17% below the
            // fence + atomicAdd + fence form.
            if (!withhold) bar_arrive(sc.bar);
            withhold = false;
            gen++;
            nsync++;
            const u64 target = gen * size;
            const u64 limit = sc.wait_ns ? sc.wait_ns : SPIN_NS;
            u64 t0 = 0, v;
            for (u32 spins = 0; (v = ld_acquire(sc.bar)) < target; spins++) {
                if ((spins & 255) == 0) {
                    const u64 now = gtimer();
                    if (t0 == 0) {
                        t0 = now;
                    } else if (now - t0 > limit) {
                        raise_err(sc.err, ST_TIMEOUT, 1);
                        break;
                    }
                }
            }
            if (v & BAR_ERR) s_err_flag = 1;
        }
        __syncthreads();
    }
};
using GridTeam = GridTeamT<true>;       // heap operations
using GridQueryTeam = GridTeamT<false>; // one query on the whole GPU

__device__ __forceinline__ u32 cluster_rank()
{
    u32 r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ u32 cluster_size()
{
    u32 r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Read a word of another CTA's shared memory in this cluster (distributed
// shared memory): `local` is the address of the same variable in this CTA.
__device__ __forceinline__ u64 dsmem_ld_u64(const u64 *local, u32 rank)
{
    u32 remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(local)), "r"(rank));
    u64 v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(remote) : "memory");
    return v;
}

// A thread-block cluster (up to 16 CTAs on one GPC) as a team: the hardware
// cluster barrier with release/acquire semantics joins it, so no software
// spin is needed.
struct ClusterTeam {
    static constexpr bool kSingle = false;
    static constexpr bool kTimed = false;
    static constexpr bool kSoftBarrier = false;
    // The hardware barrier cannot be released early, so every CTA must take
    // the same branch: read the status word itself (an error raised before a
    // barrier is seen by all after it).
    __device__ __forceinline__ bool failed() const { return read_err(sc.err) != 0; }
    Scratch sc;
    u64 nsync = 0;
    __device__ __forceinline__ u32 ncta() const { return cluster_size(); }
    __device__ __forceinline__ u32 cta() const { return cluster_rank(); }
    __device__ void init() {}
    __device__ __forceinline__ void sync()
    {
        nsync++;
        cluster_barrier();
    }
};

struct CtaTeam {
    static constexpr bool kSingle = true;
    static constexpr bool kTimed = false;
    static constexpr bool kSoftBarrier = false;
    // Only this CTA raises errors for its query.
    __device__ __forceinline__ bool failed() const { return s_err_flag != 0; }
    Scratch sc;
    u64 nsync = 0;
    __device__ __forceinline__ u32 ncta() const { return 1; }
    __device__ __forceinline__ u32 cta() const { return 0; }
    __device__ void init() {}
    __device__ __forceinline__ void sync()
    {
        nsync++;
        __syncthreads();
    }
};

// Phase timer: CTA 0's thread 0 accumulates device time per phase.
template <class Team>
struct PhaseTimer {
    Team &t;
    int slot;
    u64 t0;
    __device__ PhaseTimer(Team &tt, int s) : t(tt), slot(s), t0(0)
    {
        if constexpr (Team::kTimed)
            if (t.cta() == 0 && threadIdx.x == 0) t0 = gtimer();
    }
    __device__ ~PhaseTimer()
    {
        if constexpr (Team::kTimed)
            if (t.cta() == 0 && threadIdx.x == 0) stat_add(t.sc.stats + slot, gtimer() - t0);
    }
};

// -------------------------------------------------------- block helpers

// Exclusive block scan of v; *total receives the sum.  Contains barriers.
__device__ __forceinline__ u32 block_scan(u32 v, u32 *total, Smem &S)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u32 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        u32 y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) S.scan[warp] = x;
    __syncthreads();
    if (warp == 0) {
        u32 s = lane < NWARPS ? S.scan[lane] : 0;
        u32 inc = s;
#pragma unroll
        for (int o = 1; o < NWARPS; o <<= 1) {
            u32 y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane < NWARPS) S.scan[lane] = inc - s;
        if (lane == NWARPS - 1) S.scan[NWARPS] = inc;
    }
    __syncthreads();
    u32 r = x - v + S.scan[warp];
    *total = S.scan[NWARPS];
    __syncthreads();
    return r;
}

// Exclusive block scan of a 64-bit v (several small counters packed in
// disjoint bit fields are scanned at once); *total receives the sum.
// Contains barriers.
__device__ __forceinline__ u64 block_scan64(u64 v, u64 *total, Smem &S)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    u64 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u64 y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) S.scan64[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const u64 s0 = lane < NWARPS ? S.scan64[lane] : 0;
        u64 inc = s0;
#pragma unroll
        for (int o = 1; o < NWARPS; o <<= 1) {
            const u64 y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane < NWARPS) S.scan64[lane] = inc - s0;
        if (lane == NWARPS - 1) S.scan64[NWARPS] = inc;
    }
    __syncthreads();
    const u64 r = x - v + S.scan64[warp];
    *total = S.scan64[NWARPS];
    __syncthreads();
    return r;
}

// Sum of v over the block (all threads get it).  Contains barriers.
__device__ __forceinline__ u64 block_sum(u64 v, Smem &S)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) S.bc[8 + warp % 8] = 0;
    __syncthreads();
    if (lane == 0) atomicAdd(&S.bc[8], v);
    __syncthreads();
    u64 r = S.bc[8];
    __syncthreads();
    return r;
}

// Warp-cooperative search: pred monotone (true on [lo, ans), false on
// [ans, hi)); returns ans in every lane.  Probes 32 points per step, so a
// search over N elements costs about log_33(N) dependent global loads.

template <class Pred>
__device__ __forceinline__ u64 warp_first_false(u64 lo, u64 hi, Pred pred)
{
    const int lane = threadIdx.x & 31;
    if (lo > hi) { // an inconsistent run: report and probe nothing
        if (lane == 0 && s_err_sink) raise_err(s_err_sink, ST_CAPACITY, 20);
        return lo;
    }
    while (hi - lo > 32) {
        u64 span = hi - lo;
        u64 p = lo + ((u64)(lane + 1) * span) / 33;
        bool pr = pred(p);
        u32 m = __ballot_sync(0xffffffffu, pr);
        int c = __popc(m);
        u64 plo = __shfl_sync(0xffffffffu, p, c > 0 ? c - 1 : 0);
        u64 phi = __shfl_sync(0xffffffffu, p, c < 32 ? c : 31);
        if (c > 0) lo = plo + 1;
        if (c < 32) hi = phi;
    }
    u64 p = lo + lane;
    bool pr = (p < hi) && pred(p);
    u32 m = __ballot_sync(0xffffffffu, pr);
    return lo + __popc(m);
}

// Merge-path split: how many of the first diag elements of merge(A, B) come
// from A, ties taken from A first.
__device__ __forceinline__ u64 warp_mp_split(const u64 *A, u64 na, const u64 *B, u64 nb, u64 diag)
{
    u64 lo = diag > nb ? diag - nb : 0;
    u64 hi = diag < na ? diag : na;
    return warp_first_false(lo, hi, [&](u64 p) { return ldg_cg(A + p) <= ldg_cg(B + (diag - 1 - p)); });
}

// Number of elements <= T in sorted X[0, n).
__device__ __forceinline__ u64 warp_count_le(const u64 *X, u64 n, u64 T)
{
    if (T == INF) return n;
    return warp_first_false(0, n, [&](u64 p) { return ldg_cg(X + p) <= T; });
}

__device__ __forceinline__ u32 sm_mp_split(const u64 *A, u32 na, const u64 *B, u32 nb, u32 diag)
{
    u32 lo = diag > nb ? diag - nb : 0;
    u32 hi = diag < na ? diag : na;
    while (lo < hi) {
        u32 mid = (lo + hi) >> 1;
        if (A[mid] <= B[diag - 1 - mid])
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Shared-memory swizzle for 8-byte words: a bijection on every aligned block
// of 16 words.  Thread-contiguous chunks (thread t touching word 8t + k) and
// coalesced patterns (16 consecutive words) both land on 16 distinct bank
// pairs, so neither conflicts.
__device__ __forceinline__ u32 sw(u32 i) { return i ^ ((i >> 4) & 7); }

// Merge-path split and serial merge over runs held in the swizzled buffer W:
// A = W[sw(a0 + x)], x < na; B = W[sw(b0 + y)], y < nb.
__device__ __forceinline__ u32 sm_mp_split_sw(const u64 *W, u32 a0, u32 na, u32 b0, u32 nb, u32 diag)
{
    u32 lo = diag > nb ? diag - nb : 0;
    u32 hi = diag < na ? diag : na;
    while (lo < hi) {
        const u32 mid = (lo + hi) >> 1;
        if (W[sw(a0 + mid)] <= W[sw(b0 + diag - 1 - mid)])
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void serial_merge_sw(const u64 *W, u32 a0, u32 la, u32 b0, u32 lb, u32 a, u32 b,
                                                u64 (&it)[IPT])
{
    u64 x = a < la ? W[sw(a0 + a)] : 0, y = b < lb ? W[sw(b0 + b)] : 0;
#pragma unroll
    for (int k = 0; k < IPT; k++) {
        const bool ta = a < la && (b >= lb || x <= y);
        if (ta) {
            it[k] = x;
            a++;
            x = a < la ? W[sw(a0 + a)] : 0;
        } else {
            it[k] = b < lb ? y : INF;
            b++;
            y = b < lb ? W[sw(b0 + b)] : 0;
        }
    }
}

// Serial merge of IPT items from shared-memory runs starting at (a, b).
__device__ __forceinline__ void serial_merge(const u64 *A, u32 la, const u64 *B, u32 lb, u32 a, u32 b,
                                             u64 (&it)[IPT])
{
    u64 x = a < la ? A[a] : 0, y = b < lb ? B[b] : 0;
#pragma unroll
    for (int k = 0; k < IPT; k++) {
        bool ta = a < la && (b >= lb || x <= y);
        if (ta) {
            it[k] = x;
            a++;
            x = a < la ? A[a] : 0;
        } else {
            it[k] = b < lb ? y : INF;
            b++;
            y = b < lb ? B[b] : 0;
        }
    }
}

// Load A[a0,a1) and B[b0,b1) into S.win and merge; thread t receives items
// [t*IPT, t*IPT + IPT) of the merged tile.
__device__ __forceinline__ void tile_load_merge(const u64 *A, u64 a0, u64 a1, const u64 *B, u64 b0, u64 b1,
                                                Smem &S, u64 (&it)[IPT])
{
    if (a1 < a0 || b1 < b0 || (a1 - a0) + (b1 - b0) > (u64)TILE) { // never overrun the window
        if (threadIdx.x == 0 && s_err_sink) raise_err(s_err_sink, ST_CAPACITY, 21);
        a1 = a0;
        b1 = b0;
    }
    const u32 la = (u32)(a1 - a0), lb = (u32)(b1 - b0);
    const u32 n = la + lb;
#ifdef PBH_BULK_TILES
    // Bulk-copy variant: each run's 16-byte-aligned middle by one bulk copy
    // (cp.async.bulk, completed on an mbarrier), its odd first and last words
    // by plain loads.  A run starts at the window index with its source's
    // word parity, so aligned source words land on aligned window words
    // (the window is 16-byte aligned); sizes are even word counts.  The
    // mbarrier is initialised for each tile and invalidated after it.
    const u32 sa = la ? (u32)((reinterpret_cast<uintptr_t>(A + a0) >> 3) & 1) : 0;
    const u32 pb = lb ? (u32)((reinterpret_cast<uintptr_t>(B + b0) >> 3) & 1) : 0;
    const u32 sb = sa + la + (((sa + la) ^ pb) & 1);
    const u32 ha = la ? sa : 0, hb = lb ? pb : 0;
    const u32 ma = la > ha ? (la - ha) & ~1u : 0, mb = lb > hb ? (lb - hb) & ~1u : 0;
    const u32 bytes = 8 * (ma + mb);
    u64 *Aw = S.win + sa, *Bw = S.win + sb;
    if (threadIdx.x == 0) S.mbar_late = 0;
    if (threadIdx.x == 0 && bytes) {
        mbar_init(&S.tile_mbar); // also orders earlier generic window accesses before the copies
        fence_proxy_async_global();
        mbar_arrive_expect(&S.tile_mbar, bytes);
        if (ma) bulk_g2s(Aw + ha, A + a0 + ha, 8 * ma, &S.tile_mbar);
        if (mb) bulk_g2s(Bw + hb, B + b0 + hb, 8 * mb, &S.tile_mbar);
    }
    for (u32 i = threadIdx.x; i < la - ma; i += NT) { // head [0, ha) and tail [ha + ma, la)
        const u32 j = i < ha ? i : ma + i;
        Aw[j] = ldg_cg(A + a0 + j);
    }
    for (u32 i = threadIdx.x; i < lb - mb; i += NT) {
        const u32 j = i < hb ? i : mb + i;
        Bw[j] = ldg_cg(B + b0 + j);
    }
    __syncthreads(); // the barrier is initialised before anyone tests it
    if (bytes && !mbar_wait(&S.tile_mbar, 0)) S.mbar_late = 1;
    __syncthreads();
    if (threadIdx.x == 0 && bytes) {
        if (S.mbar_late) {
            // the copies did not land within the bound: latch the error, wait
            // once more (bounded) for them, and invalidate only if they landed
            if (s_err_sink) raise_err(s_err_sink, ST_TIMEOUT, 29);
            if (mbar_wait(&S.tile_mbar, 0)) mbar_inval(&S.tile_mbar);
        } else {
            mbar_inval(&S.tile_mbar);
        }
    }
#else
    u64 *Aw = S.win, *Bw = S.win + la;
    {
        // issue all IPT loads of this thread before using any (one round trip, not IPT)
        u64 v[IPT];
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const u32 i = threadIdx.x + k * NT;
            v[k] = i < la ? ldg_cg(A + a0 + i) : (i < n ? ldg_cg(B + b0 + (i - la)) : 0);
        }
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const u32 i = threadIdx.x + k * NT;
            if (i < n) S.win[i] = v[k];
        }
    }
    __syncthreads();
#endif
    const u32 diag = min((u32)threadIdx.x * IPT, n);
    const u32 a = sm_mp_split(Aw, la, Bw, lb, diag);
    serial_merge(Aw, la, Bw, lb, a, diag - a, it);
    __syncthreads();
}

// Write the IPT items of every thread (tile order) to out[0, n) coalesced.
__device__ __forceinline__ void tile_store(u64 *out, u32 n, const u64 (&it)[IPT], Smem &S)
{
#pragma unroll
    for (int k = 0; k < IPT; k++) S.win[sw(threadIdx.x * IPT + k)] = it[k];
    __syncthreads();
    for (u32 i = threadIdx.x; i < n; i += NT) out[i] = S.win[sw(i)];
    __syncthreads();
}

// Validity + dedup flags of this thread's items: item x at tile position p
// (< n) survives iff cur[key(x)] == x (it is the live word of its key) and
// x differs from the element before it in merged order.  The predecessor of
// the tile's first element is (pv, hp).  Returns the flag byte.
__device__ __forceinline__ u32 tile_flags(const u64 (&it)[IPT], u32 n, u64 pv, bool hp, const u64 *cur,
                                          u64 kmask, Smem &S)
{
    const u64 kspace = S.hs.key_space;
    S.last[threadIdx.x] = it[IPT - 1];
    __syncthreads();
    const u32 my0 = threadIdx.x * IPT;
    u64 p = threadIdx.x == 0 ? pv : S.last[threadIdx.x - 1];
    bool h = threadIdx.x == 0 ? hp : true;
    u64 cv[IPT];
#pragma unroll
    for (int k = 0; k < IPT; k++) {
        cv[k] = ~it[k]; // "not valid" unless the key is in range
        if (my0 + k < n) {
            const u64 key = it[k] & kmask;
            if (key < kspace)
                cv[k] = ldg_cg(cur + key);
            else if (s_err_sink)
                raise_err(s_err_sink, ST_CAPACITY, 23);
        }
    }
    u32 flags = 0;
#pragma unroll
    for (int k = 0; k < IPT; k++) {
        if (my0 + k < n) {
            bool ok = (cv[k] == it[k]) && (!h || it[k] != p);
            flags |= (u32)ok << k;
            p = it[k];
            h = true;
        }
    }
    __syncthreads();
    return flags;
}

// Compact the flagged items of the tile into S.keep[0, total) in order.
__device__ __forceinline__ u32 tile_compact(const u64 (&it)[IPT], u32 flags, Smem &S)
{
    u32 total;
    u32 excl = block_scan(__popc(flags), &total, S);
    u32 j = excl;
#pragma unroll
    for (int k = 0; k < IPT; k++)
        if (flags >> k & 1) S.keep[sw(j++)] = it[k];
    __syncthreads();
    return total;
}

// ------------------------------------------------------------ merges

struct MergeOut {
    u64 kept;  // elements written
    u64 a_end; // elements of A consumed (split of the D-th output)
    u64 last;  // the D-th merged element (valid or not), the predecessor of a continuation
    bool has_last;
};

// Merge the first D outputs of merge(A, B) (two sorted runs), drop every
// element that is not the live word of its key or equals its predecessor
// (DeleteDuplicates of Algorithm 1 under the validity reading), and write the
// survivors compacted and sorted to out.  (pred0, has_pred0) is the element
// before the first output, if any.  Ends with a team barrier.
template <class Team>
__device__ __forceinline__ MergeOut merge_filter_impl(Team &t, Smem &S, const u64 *A, u64 na, const u64 *B,
                                                      u64 nb, u64 D, u64 *out, const u64 *cur, u64 kmask,
                                                      u64 pred0, bool has_pred0)
{
    const u32 tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (D == 0) return MergeOut{0, 0, pred0, has_pred0};
    if (D > na + nb) { // inconsistent state: refuse rather than read out of bounds
        raise_err(t.sc.err, ST_CAPACITY, 2);
        return MergeOut{0, 0, pred0, has_pred0};
    }
    if constexpr (Team::kSingle) {
        u64 base = 0, a0 = 0, pv = pred0;
        bool hp = has_pred0;
        for (u64 d0 = 0; d0 < D; d0 += TILE) {
            const u64 d1 = min(d0 + (u64)TILE, D);
            if (warp == 0) {
                u64 a1 = warp_mp_split(A, na, B, nb, d1);
                if (lane == 0) S.bc[0] = a1;
            }
            __syncthreads();
            const u64 a1 = S.bc[0];
            u64 it[IPT];
            tile_load_merge(A, a0, a1, B, d0 - a0, d1 - a1, S, it);
            const u32 n = (u32)(d1 - d0);
            u32 flags = tile_flags(it, n, pv, hp, cur, kmask, S);
            const u32 kept = tile_compact(it, flags, S);
            for (u32 i = tid; i < kept; i += NT) out[base + i] = S.keep[sw(i)];
            const u32 my0 = tid * IPT;
            if (n - 1 >= my0 && n - 1 < my0 + IPT) S.bc[1] = it[n - 1 - my0];
            __syncthreads();
            pv = S.bc[1];
            hp = true;
            base += kept;
            a0 = a1;
            __syncthreads();
        }
        return MergeOut{base, a0, pv, hp};
    } else {
        const u64 P = t.ncta(), c = t.cta();
        const u64 ntiles = (D + TILE - 1) / TILE;
        const u64 per = (ntiles + P - 1) / P;
        const u64 j0 = min(c * per, ntiles), j1 = min(j0 + per, ntiles);
        const bool single = (per == 1);
        u64 local = 0;
        u32 keep_n = 0;
        if (j0 < j1) {
            if (warp == 0) {
                u64 a = warp_mp_split(A, na, B, nb, j0 * TILE);
                if (lane == 0) S.bc[0] = a;
            } else if (warp == 1) {
                u64 a = warp_mp_split(A, na, B, nb, min(j1 * (u64)TILE, D));
                if (lane == 0) S.bc[2] = a;
            }
            __syncthreads();
            u64 a0 = S.bc[0];
            const u64 aend = S.bc[2];
            if (tid == 0 && !single) t.sc.splits[j0] = a0;
            for (u64 j = j0; j < j1; j++) {
                const u64 d0 = j * TILE, d1 = min(d0 + (u64)TILE, D);
                // the split after this tile goes to its own slot: S.bc[0] and
                // S.bc[2] may still be read (a0, aend) in the first iteration
                if (j + 1 < j1 && warp == 0) {
                    u64 a = warp_mp_split(A, na, B, nb, d1);
                    if (lane == 0) S.bc[1] = a;
                }
                if (tid == 0) {
                    u64 pv;
                    bool hp;
                    if (d0 == 0) {
                        pv = pred0;
                        hp = has_pred0;
                    } else {
                        const u64 b0 = d0 - a0;
                        const u64 xa = a0 > 0 ? ldg_cg(A + a0 - 1) : 0;
                        const u64 xb = b0 > 0 ? ldg_cg(B + b0 - 1) : 0;
                        pv = a0 == 0 ? xb : (b0 == 0 ? xa : (xa > xb ? xa : xb));
                        hp = true;
                    }
                    S.bc[3] = pv;
                    S.bc[4] = hp;
                }
                __syncthreads();
                const u64 a1 = j + 1 < j1 ? S.bc[1] : aend;
                const u64 pv = S.bc[3];
                const bool hp = S.bc[4] != 0;
                if (tid == 0 && !single) t.sc.splits[j + 1] = a1;
                u64 it[IPT];
                tile_load_merge(A, a0, a1, B, d0 - a0, d1 - a1, S, it);
                const u32 n = (u32)(d1 - d0);
                const u32 flags = tile_flags(it, n, pv, hp, cur, kmask, S);
                if (single) {
                    keep_n = tile_compact(it, flags, S);
                    local += keep_n;
                } else {
                    t.sc.bits[d0 / 8 + tid] = (unsigned char)flags;
                    u32 tot;
                    block_scan(__popc(flags), &tot, S);
                    local += tot;
                }
                if (j + 1 == ntiles) {
                    const u32 my0 = tid * IPT;
                    if (n - 1 >= my0 && n - 1 < my0 + IPT) {
                        t.sc.res[1] = a1;
                        t.sc.res[2] = it[n - 1 - my0];
                    }
                }
                a0 = a1;
                __syncthreads();
            }
        }
        if (tid == 0) t.sc.partials[c] = local;
        t.sync();
        // Read the results of pass 1 before the closing barrier: once a CTA
        // passes it, the next merge may overwrite res and partials.
        const u64 r_aend = ldg_cg(t.sc.res + 1), r_last = ldg_cg(t.sc.res + 2);
        u64 excl = 0, total = 0;
        for (u64 i = tid; i < P; i += NT) {
            u64 v = ldg_cg(t.sc.partials + i);
            total += v;
            if (i < c) excl += v;
        }
        if (D < (1ull << 32)) { // one reduction for both sums
            const u64 both = block_sum((total << 32) | excl, S);
            total = both >> 32;
            excl = both & 0xffffffffull;
        } else {
            total = block_sum(total, S);
            excl = block_sum(excl, S);
        }
        if (j0 < j1) {
            if (single) {
                for (u32 i = tid; i < keep_n; i += NT) out[excl + i] = S.keep[sw(i)];
            } else {
                u64 base = excl;
                for (u64 j = j0; j < j1; j++) {
                    const u64 d0 = j * TILE, d1 = min(d0 + (u64)TILE, D);
                    const u64 a0 = ldg_cg(t.sc.splits + j), a1 = ldg_cg(t.sc.splits + j + 1);
                    u64 it[IPT];
                    tile_load_merge(A, a0, a1, B, d0 - a0, d1 - a1, S, it);
                    const u32 flags = t.sc.bits[d0 / 8 + tid];
                    const u32 kept = tile_compact(it, flags, S);
                    for (u32 i = tid; i < kept; i += NT) out[base + i] = S.keep[sw(i)];
                    base += kept;
                    __syncthreads();
                }
            }
        }
        t.sync();
        return MergeOut{total, r_aend, r_last, true};
    }
}
// Multi-CTA teams call the general merges, the team sort, Empty and Fill
// out of line (the *_out wrappers): on the SSSP path they run in few rounds,
// and inlined into the round loop they raised its register pressure past
// 255 registers (spills in the hot loop).  One-CTA teams, whose queries
// merge often, keep them inline.
template <class Team>
__noinline__ __device__ MergeOut merge_filter_out(Team &t, Smem &S, const u64 *A, u64 na, const u64 *B, u64 nb,
                                                  u64 D, u64 *out, const u64 *cur, u64 kmask, u64 pred0,
                                                  bool has_pred0)
{
    return merge_filter_impl<Team>(t, S, A, na, B, nb, D, out, cur, kmask, pred0, has_pred0);
}
template <class Team>
__device__ __forceinline__ MergeOut merge_filter(Team &t, Smem &S, const u64 *A, u64 na, const u64 *B, u64 nb,
                                                 u64 D, u64 *out, const u64 *cur, u64 kmask, u64 pred0,
                                                 bool has_pred0)
{
    if constexpr (Team::kSingle)
        return merge_filter_impl<Team>(t, S, A, na, B, nb, D, out, cur, kmask, pred0, has_pred0);
    else
        return merge_filter_out<Team>(t, S, A, na, B, nb, D, out, cur, kmask, pred0, has_pred0);
}

// Plain merge of two sorted runs into out[0, na + nb).  Ends with a team barrier.
template <class Team>
__device__ __forceinline__ void merge_plain_impl(Team &t, Smem &S, const u64 *A, u64 na, const u64 *B, u64 nb, u64 *out)
{
    const u32 tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const u64 n = na + nb;
    const u64 ntiles = (n + TILE - 1) / TILE;
    for (u64 j = t.cta(); j < ntiles; j += t.ncta()) {
        const u64 d0 = j * TILE, d1 = min(d0 + (u64)TILE, n);
        if (warp == 0) {
            u64 a = warp_mp_split(A, na, B, nb, d0);
            if (lane == 0) S.bc[0] = a;
        } else if (warp == 1) {
            u64 a = warp_mp_split(A, na, B, nb, d1);
            if (lane == 0) S.bc[1] = a;
        }
        __syncthreads();
        const u64 a0 = S.bc[0], a1 = S.bc[1];
        u64 it[IPT];
        tile_load_merge(A, a0, a1, B, d0 - a0, d1 - a1, S, it);
        tile_store(out + d0, (u32)(d1 - d0), it, S);
    }
    t.sync();
}
template <class Team>
__noinline__ __device__ void merge_plain_out(Team &t, Smem &S, const u64 *A, u64 na, const u64 *B, u64 nb, u64 *out)
{
    merge_plain_impl<Team>(t, S, A, na, B, nb, out);
}
template <class Team>
__device__ __forceinline__ void merge_plain(Team &t, Smem &S, const u64 *A, u64 na, const u64 *B, u64 nb, u64 *out)
{
    if constexpr (Team::kSingle)
        merge_plain_impl<Team>(t, S, A, na, B, nb, out);
    else
        merge_plain_out<Team>(t, S, A, na, B, nb, out);
}

// Team copy src[0, n) -> dst[0, n) (non-overlapping).  Ends with a team barrier.
template <class Team>
__device__ void team_copy(Team &t, const u64 *src, u64 n, u64 *dst)
{
    const u64 stride = (u64)t.ncta() * NT;
    for (u64 i = (u64)t.cta() * NT + threadIdx.x; i < n; i += stride) dst[i] = ldg_cg(src + i);
    t.sync();
}

// ------------------------------------------------------------- sorting

__device__ __forceinline__ void cas(u64 &a, u64 &b)
{
    u64 x = a < b ? a : b, y = a < b ? b : a;
    a = x;
    b = y;
}

// Bitonic sort of the 256 words a warp holds, 8 per lane, lane-major (lane l
// holds positions 8l .. 8l+7): compare-exchanges within a lane use registers,
// across lanes one shuffle per word.  No shared memory, no block barrier.
__device__ __forceinline__ void warp_bitonic256(u64 (&it)[IPT])
{
    const u32 lane = threadIdx.x & 31;
#pragma unroll
    for (u32 size = 2; size <= 256; size <<= 1) {
#pragma unroll
        for (u32 stride = size / 2; stride > 0; stride >>= 1) {
            if (stride >= IPT) {
                const u32 lm = stride / IPT;                 // partner lane distance
                const bool asc = ((lane * IPT) & size) == 0; // direction of this bitonic block
                const bool keep_min = ((lane & lm) == 0) == asc;
#pragma unroll
                for (int k = 0; k < IPT; k++) {
                    const u64 o = __shfl_xor_sync(0xffffffffu, it[k], lm);
                    it[k] = keep_min ? (o < it[k] ? o : it[k]) : (o > it[k] ? o : it[k]);
                }
            } else {
#pragma unroll
                for (int k = 0; k < IPT; k++) {
                    const int p = k ^ (int)stride;
                    if (p > k) {
                        const bool asc = ((lane * IPT + k) & size) == 0;
                        const u64 x = it[k], y = it[p];
                        const bool swp = asc ? (x > y) : (x < y);
                        it[k] = swp ? y : x;
                        it[p] = swp ? x : y;
                    }
                }
            }
        }
    }
}

// Sort n <= TILE words of g_in into g_out with one CTA: a register bitonic
// sort per warp (256 words), then merge-path rounds in swizzled shared memory
// (256 -> 512 -> 1024 -> 2048).  With `gather`, g_in holds keys and the
// sorted words are gather[key].
__device__ inline void block_sort_tile(const u64 *g_in, u64 *g_out, u32 n, Smem &S, const u64 *gather)
{
    {
        u64 v[IPT];
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const u32 i = threadIdx.x + k * NT;
            v[k] = i < n ? ldg_cg(g_in + i) : INF;
        }
        if (gather) {
#pragma unroll
            for (int k = 0; k < IPT; k++) {
                const u32 i = threadIdx.x + k * NT;
                if (i < n) v[k] = ldg_cg(gather + v[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < IPT; k++) S.win[sw(threadIdx.x + k * NT)] = v[k];
    }
    __syncthreads();
    u64 it[IPT];
#pragma unroll
    for (int k = 0; k < IPT; k++) it[k] = S.win[sw(threadIdx.x * IPT + k)];
    warp_bitonic256(it);
    for (u32 w = 32 * IPT; w < TILE; w *= 2) {
        __syncthreads();
#pragma unroll
        for (int k = 0; k < IPT; k++) S.win[sw(threadIdx.x * IPT + k)] = it[k];
        __syncthreads();
        const u32 pos = threadIdx.x * IPT;
        const u32 pair0 = (pos / (2 * w)) * (2 * w);
        const u32 diag = pos - pair0;
        const u32 a = sm_mp_split_sw(S.win, pair0, w, pair0 + w, w, diag);
        serial_merge_sw(S.win, pair0, w, pair0 + w, w, a, diag - a, it);
    }
    __syncthreads();
    tile_store(g_out, n, it, S);
}

// Rank sort of n <= TILE words with the team: every CTA stages all
// n words in shared memory; each warp takes elements in turn and its lanes
// count, in parallel, the words that precede the element (ties broken by
// position, so the ranks are a permutation); the element is written straight
// to its rank.  One team barrier, no merge passes.  With `gather`, src holds
// keys and the sorted words are gather[key].  Ends with a team barrier.
template <class Team>
__device__ void team_rank_sort(Team &t, Smem &S, const u64 *src, u32 n, u64 *dst, const u64 *gather)
{
    {
        u64 v[IPT];
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const u32 i = threadIdx.x + k * NT;
            v[k] = i < n ? ldg_cg(src + i) : 0;
        }
        if (gather) {
#pragma unroll
            for (int k = 0; k < IPT; k++) {
                const u32 i = threadIdx.x + k * NT;
                if (i < n) v[k] = ldg_cg(gather + v[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const u32 i = threadIdx.x + k * NT;
            if (i < n) S.win[i] = v[k];
        }
    }
    __syncthreads();
    const u32 lane = threadIdx.x & 31;
    const u32 gw = t.cta() * NWARPS + (threadIdx.x >> 5), nw = t.ncta() * NWARPS;
    for (u32 e = gw; e < n; e += nw) {
        const u64 x = S.win[e];
        u32 c = 0;
        for (u32 j = lane; j < n; j += 32) {
            const u64 y = S.win[j];
            c += (y < x) || (y == x && j < e);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) dst[c] = x;
    }
    t.sync();
}

// Sort src[0, n) with the team; tmp is a second buffer of n words.  Returns
// the buffer that holds the result.  Ends with a team barrier.
template <class Team>
__device__ __forceinline__ u64 *team_sort_impl(Team &t, Smem &S, u64 *src, u64 n, u64 *tmp, const u64 *gather = nullptr)
{
    const u32 tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const u64 ntiles = (n + TILE - 1) / TILE;
    for (u64 j = t.cta(); j < ntiles; j += t.ncta())
        block_sort_tile(src + j * TILE, tmp + j * TILE, (u32)min((u64)TILE, n - j * TILE), S, gather);
    t.sync();
    u64 *a = tmp, *b = src;
    for (u64 run = TILE; run < n; run *= 2) {
        for (u64 j = t.cta(); j < ntiles; j += t.ncta()) {
            const u64 d0 = j * TILE;
            const u64 pair0 = (d0 / (2 * run)) * (2 * run);
            const u64 na = min(run, n - pair0);
            const u64 nb = min(run, n - pair0 - na);
            const u64 ld0 = d0 - pair0, ld1 = min(ld0 + (u64)TILE, na + nb);
            const u64 *A = a + pair0, *B = A + na;
            if (warp == 0) {
                u64 s = warp_mp_split(A, na, B, nb, ld0);
                if (lane == 0) S.bc[0] = s;
            } else if (warp == 1) {
                u64 s = warp_mp_split(A, na, B, nb, ld1);
                if (lane == 0) S.bc[1] = s;
            }
            __syncthreads();
            const u64 s0 = S.bc[0], s1 = S.bc[1];
            u64 it[IPT];
            tile_load_merge(A, s0, s1, B, ld0 - s0, ld1 - s1, S, it);
            tile_store(b + d0, (u32)(ld1 - ld0), it, S);
        }
        t.sync();
        u64 *x = a;
        a = b;
        b = x;
    }
    return a;
}
template <class Team>
__noinline__ __device__ u64 *team_sort_out(Team &t, Smem &S, u64 *src, u64 n, u64 *tmp, const u64 *gather)
{
    return team_sort_impl<Team>(t, S, src, n, tmp, gather);
}
template <class Team>
__device__ __forceinline__ u64 *team_sort(Team &t, Smem &S, u64 *src, u64 n, u64 *tmp, const u64 *gather = nullptr)
{
    if constexpr (Team::kSingle)
        return team_sort_impl<Team>(t, S, src, n, tmp, gather);
    else
        return team_sort_out<Team>(t, S, src, n, tmp, gather);
}

// ------------------------------------------------------------ the heap

__device__ __forceinline__ void leader_sync() { __syncthreads(); }
#define LEADER if (threadIdx.x == 0)

// Is anything stored at a level deeper than i?
__device__ __forceinline__ bool deeper_nonempty(const HeapState &hs, int i)
{
    for (int j = i + 1; j < (int)hs.q; j++)
        if (hs.L[j].blen || hs.L[j].slen) return true;
    return false;
}

template <class Team>
__device__ __forceinline__ u64 team_count_le(Team &t, Smem &S, const u64 *X, u64 n, u64 T)
{
    if (T == INF) return n;
    if ((threadIdx.x >> 5) == 0) {
        u64 r = warp_count_le(X, n, T);
        if ((threadIdx.x & 31) == 0) S.bc[5] = r;
    }
    __syncthreads();
    u64 r = S.bc[5];
    __syncthreads();
    return r;
}

template <class Team>
__device__ __forceinline__ u64 team_load(Smem &S, const u64 *p)
{
    LEADER S.bc[6] = ldg_cg(p);
    __syncthreads();
    u64 v = S.bc[6];
    __syncthreads();
    return v;
}

template <class Team>
__device__ void empty_level(Team &t, Smem &S, int i);
template <class Team>
__device__ void empty_split(Team &t, Smem &S, int i, u64 *outB, u64 ns, u64 nb, u64 total);

// Empty(S_i) (first half of Algorithm 1): merge S_i into B_i, drop stale and
// duplicate elements, keep the elements <= T_i up to capacity (re-selecting
// T_i as the capacity-th smallest if more remain), and merge the rest into
// S_{i+1}.  At the last level T is unbounded; overflow there is a capacity
// error.
template <class Team>
__device__ __forceinline__ void empty_level_once_impl(Team &t, Smem &S, int i)
{
    HeapState &hs = S.hs;
    Level &L = hs.L[i];
    const u64 *Sr = L.S[L.ssel] + L.shead, *Br = L.B[L.bsel] + L.bhead;
    const u64 ns = L.slen, nb = L.blen;
    u64 *outB = L.B[L.bsel ^ 1];
    if (ns + nb > L.bufB || L.shead + ns > L.bufS || L.bhead + nb > L.bufB) {
        raise_err(t.sc.err, ST_CAPACITY, 25);
        return;
    }
    MergeOut mo = merge_filter(t, S, Sr, ns, Br, nb, ns + nb, outB, hs.cur, hs.keymask, 0, false);
    empty_split(t, S, i, outB, ns, nb, mo.kept);
}
template <class Team>
__noinline__ __device__ void empty_level_once_out(Team &t, Smem &S, int i)
{
    empty_level_once_impl<Team>(t, S, i);
}
template <class Team>
__device__ __forceinline__ void empty_level_once(Team &t, Smem &S, int i)
{
    if constexpr (Team::kSingle)
        empty_level_once_impl<Team>(t, S, i);
    else
        empty_level_once_out<Team>(t, S, i);
}

// Second part of Empty(S_i), after the merged, filtered run of total
// elements was written to outB (the spare B_i buffer): keep what is <= T_i
// up to capacity, push the rest into S_{i+1}, switch B_i to outB.
template <class Team>
__device__ void empty_split(Team &t, Smem &S, int i, u64 *outB, u64 ns, u64 nb, u64 total)
{
    HeapState &hs = S.hs;
    Level &L = hs.L[i];
    const u64 Ti = L.T, capB = L.capB;
    const bool last = (i + 1 == (int)hs.q);
    const u64 cle = team_count_le(t, S, outB, total, Ti);
    const u64 kept = cle < capB ? cle : capB;
    u64 newT = Ti;
    if (cle > capB) newT = team_load<Team>(S, outB + capB - 1);
    if (total > kept && last) {
        raise_err(t.sc.err, ST_CAPACITY, 4);
        return;
    }
    if (total > kept && hs.L[i + 1].slen + (total - kept) > hs.L[i + 1].bufS) {
        raise_err(t.sc.err, ST_CAPACITY, 3); // cannot happen under the schedule; never overrun the buffer
        return;
    }
    if (total > kept) {
        Level &N = hs.L[i + 1];
        u64 *outS = N.S[N.ssel ^ 1];
        merge_plain(t, S, N.S[N.ssel] + N.shead, N.slen, outB + kept, total - kept, outS);
        LEADER
        {
            N.ssel ^= 1;
            N.shead = 0;
            N.slen += total - kept;
        }
    }
    LEADER
    {
        L.bsel ^= 1;
        L.bhead = 0;
        L.blen = kept;
        L.T = newT;
        L.slen = 0;
        L.shead = 0;
        if (t.cta() == 0) {
            stat_add(t.sc.stats + STAT_STALE, ns + nb - total);
            stat_add(t.sc.stats + STAT_MERGED, ns + nb);
        }
    }
    __syncthreads();
}

// BulkUpdate sort fused with Empty(S_0), for batches whose words are all live
// and pairwise distinct with distinct keys: SSSP stages each improved vertex
// once per round and gathers its final word here, so no staged word is stale,
// none repeats, and none equals a word already in B_0 (a key's word only
// falls).  The merged output is then merge(sorted batch, live part of B_0),
// the same run Empty writes after DeleteDuplicates.
//
// B_0 is cut into one fixed slice per CTA; the slice [b0, b1) owns the batch
// words in [B_0[b0], B_0[b1]).  Before the single counting barrier every CTA
// loads its slice and checks its validity, ranks its share of the batch
// (writing the sorted batch to U[1]), and counts the batch words below its
// two boundaries, so its output count is known; after it, the CTA loads its
// batch range from U[1] and scatters both runs to their merged positions.
// The batch size n (the staging count) is loaded in the same round trip as
// the staged ids, which are read speculatively up to min(TILE, d) (entries
// past n are left from earlier rounds and never used).  Requires a slice of
// at most TILE.  Returns FUSED_NO (n = 0 or n > TILE: nothing was done, use
// the general path), FUSED_ERR (a capacity error was latched) or FUSED_OK
// with the merged count in *total.  *n_out receives n in every case.
enum : int { FUSED_NO = 0, FUSED_OK = 1, FUSED_ERR = 2 };

template <class Team>
__device__ int empty0_fused(Team &t, Smem &S, u64 *n_out, u64 *total_out)
{
    HeapState &hs = S.hs;
    Level &L = hs.L[0];
    const u32 tid = threadIdx.x, lane = tid & 31;
    const u64 nb = L.blen;
    const u64 *Br = L.B[L.bsel] + L.bhead;
    u64 *outB = L.B[L.bsel ^ 1];
    const u64 *cur = hs.cur, kmask = hs.keymask, kspace = hs.key_space;
    const u64 P = t.ncta(), c = t.cta();
    const u64 per = (nb + P - 1) / P;
    const u64 b0 = min(c * per, nb), b1 = min(b0 + per, nb);
    const u32 nbs = (u32)(b1 - b0);
    const u64 *U0 = hs.U[0];
    u64 *sorted = hs.U[1];
    const u32 nspec = (u32)min((u64)TILE, hs.d); // U[0] holds d words
    // 1. the batch size, the staged ids (speculatively), the slice and its
    // boundaries in one round of loads; then the batch words (gathered by
    // key) into win and the slice into registers (striped)
    u64 bw[IPT];
    const u64 lo_w = (c > 0 && b0 < nb) ? ldg_cg(Br + b0) : 0;
    const u64 hi_w = b1 < nb ? ldg_cg(Br + b1) : 0;
    u32 n;
    {
        u64 v[IPT];
        if (tid == 0) S.bc[6] = ldg_cg(t.sc.ucount);
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const u32 i = tid + k * NT;
            v[k] = i < nspec ? ldg_cg(U0 + i) : 0;
            bw[k] = i < nbs ? ldg_cg(Br + b0 + i) : INF;
        }
        __syncthreads();
        const u64 n64 = S.bc[6];
        *n_out = n64;
        if (n64 == 0 || n64 > nspec) return FUSED_NO; // uniform
        if (n64 + nb > L.bufB || L.bhead + nb > L.bufB) {
            raise_err(t.sc.err, ST_CAPACITY, 25);
            return FUSED_ERR;
        }
        n = (u32)n64;
        u64 cv[IPT];
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const u32 i = tid + k * NT;
            if (i < n) {
                if (v[k] < kspace) {
                    v[k] = ldg_cg(cur + v[k]);
                } else {
                    raise_err(t.sc.err, ST_CAPACITY, 23);
                    v[k] = INF;
                }
            }
            cv[k] = ~bw[k];
            if (i < nbs) {
                const u64 key = bw[k] & kmask;
                if (key < kspace)
                    cv[k] = ldg_cg(cur + key);
                else
                    raise_err(t.sc.err, ST_CAPACITY, 23);
            }
        }
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const u32 i = tid + k * NT;
            if (i < n) S.win[i] = v[k];
            if (i < nbs && cv[k] != bw[k]) bw[k] = INF; // stale: dropped
            if (i < nbs) S.keep[sw(i)] = bw[k];
        }
    }
    __syncthreads();
    PBH_PROBE(t, 5); // batch ids, their words, the B_0 slice and its validity
    // 2. rank this team's share of the batch into U[1]
    {
        const u32 gw = (u32)c * NWARPS + (tid >> 5), nw = (u32)P * NWARPS;
        for (u32 e = gw; e < n; e += nw) {
            const u64 x = S.win[e];
            u32 r = 0;
            for (u32 j = lane; j < n; j += 32) r += S.win[j] < x;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
            if (lane == 0) sorted[r] = x;
        }
    }
    PBH_PROBE(t, 6); // rank sort of this CTA's share of the batch
    // 3. this CTA's batch range [lo, hi) (words below each slice boundary)
    // and 4. the live slice words compacted into keep[sw(0..vb)): one scan of
    // (words below the low boundary, below the high one, live slice words),
    // packed in 21-bit fields (each count <= TILE)
    u64 lo, hi;
    u32 vb;
    {
        u32 clo = 0, chi = 0;
        for (u32 j = tid; j < n; j += NT) {
            const u64 x = S.win[j];
            clo += x < lo_w;
            chi += x < hi_w;
        }
        u64 it[IPT];
        u32 cnt = 0;
#pragma unroll
        for (int k = 0; k < IPT; k++) {
            const u32 i = tid * IPT + k;
            it[k] = i < nbs ? S.keep[sw(i)] : INF;
            cnt += it[k] != INF;
        }
        constexpr u64 F21 = (1ull << 21) - 1;
        u64 tot;
        const u64 ex = block_scan64(((u64)clo << 42) | ((u64)chi << 21) | cnt, &tot, S); // its barriers order
        u32 j = (u32)(ex & F21);                                                          // the reads above
#pragma unroll                                                                            // before the writes
        for (int k = 0; k < IPT; k++)
            if (it[k] != INF) S.keep[sw(j++)] = it[k];
        vb = (u32)(tot & F21);
        const u64 nlo = tot >> 42, nhi = (tot >> 21) & F21;
        lo = (c == 0) ? 0 : (b0 < nb ? nlo : n);
        hi = (b1 < nb) ? nhi : n;
        if (c > 0 && b0 >= nb) hi = n;
        if (hi < lo) { // the slices' boundaries are sorted, so this cannot happen
            raise_err(t.sc.err, ST_CAPACITY, 26);
            hi = lo;
        }
    }
    if (tid == 0) t.sc.partials[c] = vb + (hi - lo);
    PBH_PROBE(t, 7); // boundary counts, slice compaction
    PBH_SPAN_END(t, 16); // relax barrier to the counting barrier, per CTA (sum, max)
    t.sync();
    PBH_SPAN_BEGIN();
    PBH_PROBE(t, 8); // counting barrier
    // 5. output offset, then scatter both runs to their merged positions (the
    // batch range is issued first: it does not depend on the partials)
    const u32 ns = (u32)(hi - lo);
    u64 sv[IPT];
#pragma unroll
    for (int k = 0; k < IPT; k++) {
        const u32 i = tid + k * NT;
        sv[k] = i < ns ? ldg_cg(sorted + lo + i) : 0;
    }
    u64 excl = 0, total = 0;
    for (u64 i = tid; i < P; i += NT) {
        const u64 x = ldg_cg(t.sc.partials + i);
        total += x;
        if (i < c) excl += x;
    }
    // every CTA read the batch size before this barrier: the next round may count again
    if (c == 0 && tid == 0) *t.sc.ucount = 0;
#pragma unroll
    for (int k = 0; k < IPT; k++) {
        const u32 i = tid + k * NT;
        if (i < ns) S.win[i] = sv[k];
    }
    {
        // one reduction for both sums (each below 2^32: at most 4d words)
        const u64 both = block_sum((total << 32) | excl, S);
        total = both >> 32;
        excl = both & 0xffffffffull;
    }
    PBH_PROBE(t, 9); // partial counts, this CTA's sorted batch range
    u64 *out = outB + excl;
    for (u32 i = tid; i < ns; i += NT) { // batch word: its index + live slice words below it
        const u64 x = S.win[i];
        u32 a = 0, b = vb;
        while (a < b) {
            const u32 m = (a + b) >> 1;
            if (S.keep[sw(m)] < x)
                a = m + 1;
            else
                b = m;
        }
        out[i + a] = x;
    }
    for (u32 j = tid; j < vb; j += NT) { // slice word: its index + batch words below it
        const u64 y = S.keep[sw(j)];
        u32 a = 0, b = ns;
        while (a < b) {
            const u32 m = (a + b) >> 1;
            if (S.win[m] < y)
                a = m + 1;
            else
                b = m;
        }
        out[j + a] = y;
    }
    PBH_PROBE(t, 10); // scatter of both runs
    PBH_SPAN_END(t, 18); // counting barrier to the closing barrier, per CTA (sum, max)
    t.sync();
    PBH_PROBE(t, 11); // closing barrier
    *total_out = total;
    return FUSED_OK;
}

// Empty level i, then empty any deeper signal buffer pushed over capacity.
template <class Team>
__device__ void empty_level(Team &t, Smem &S, int i)
{
    empty_level_once(t, S, i);
    for (int j = i + 1; j < (int)S.hs.q && !t.failed(); j++) {
        if (S.hs.L[j].slen <= S.hs.L[j].capS) break;
        empty_level_once(t, S, j);
    }
}

// Fill(B_i) (second half of Algorithm 1): pull the smallest live elements of
// level i+1 into B_i until it holds capB_i.  The candidates are B_{i+1} and
// the part of S_{i+1} that is <= T_{i+1} (the rest of S_{i+1} belongs deeper);
// runs are sorted, so the pulled elements are a merged prefix and are larger
// than everything already in B_i: they are appended.  T_i becomes the last
// pulled element, or T_{i+1} if level i+1 ran out of candidates.
template <class Team>
__device__ __forceinline__ void fill_level_impl(Team &t, Smem &S, int i)
{
    HeapState &hs = S.hs;
    Level &L = hs.L[i];
    Level &N = hs.L[i + 1];
    u64 want = L.capB > L.blen ? L.capB - L.blen : 0;
    if (want == 0) return;
    if (L.bhead + L.blen + want > L.bufB) { // make room: move B_i to the start of the other buffer
        team_copy(t, L.B[L.bsel] + L.bhead, L.blen, L.B[L.bsel ^ 1]);
        LEADER
        {
            L.bsel ^= 1;
            L.bhead = 0;
        }
        __syncthreads();
    }
    u64 sle = team_count_le(t, S, N.S[N.ssel] + N.shead, N.slen, N.T);
    u64 pv = 0;
    bool hp = false;
    bool got_any = false;
    while (want > 0 && !t.failed()) {
        // Snapshot the shared control state into registers: the leader updates
        // it below within this same barrier interval, so no thread may read
        // it again after the merge (every decision must be CTA-uniform).
        const u64 nblen = N.blen;
        const u64 avail = nblen + sle;
        if (avail == 0) break;
        const u64 D = want < avail ? want : avail;
        u64 *dst = L.B[L.bsel] + L.bhead + L.blen;
        MergeOut mo = merge_filter(t, S, N.B[N.bsel] + N.bhead, nblen, N.S[N.ssel] + N.shead, sle, D, dst,
                                   hs.cur, hs.keymask, pv, hp);
        pv = mo.last;
        hp = mo.has_last;
        const u64 ca = mo.a_end, cb = D - mo.a_end;
        if (ca > nblen || cb > sle || mo.kept > want) { // uniform: registers only
            raise_err(t.sc.err, ST_CAPACITY, 5);        // inconsistent merge result: stop instead of looping
            break;
        }
        if (t.failed()) break; // raised inside the merge, before its closing barrier
        sle -= cb;
        want -= mo.kept;
        got_any |= mo.kept > 0;
        LEADER
        {
            N.bhead += ca;
            N.blen -= ca;
            N.shead += cb;
            N.slen -= cb;
            L.blen += mo.kept;
            if (t.cta() == 0) {
                stat_add(t.sc.stats + STAT_STALE, D - mo.kept);
                stat_add(t.sc.stats + STAT_MERGED, D);
            }
        }
        __syncthreads();
    }
    u64 newT;
    if (want == 0)
        newT = team_load<Team>(S, L.B[L.bsel] + L.bhead + L.blen - 1);
    else
        newT = N.T;
    (void)got_any;
    LEADER L.T = newT;
    __syncthreads();
}
template <class Team>
__noinline__ __device__ void fill_level_out(Team &t, Smem &S, int i)
{
    fill_level_impl<Team>(t, S, i);
}
template <class Team>
__device__ __forceinline__ void fill_level(Team &t, Smem &S, int i)
{
    if constexpr (Team::kSingle)
        fill_level_impl<Team>(t, S, i);
    else
        fill_level_out<Team>(t, S, i);
}

template <class Team>
__device__ void resolve_fill(Team &t, Smem &S, int i);

// Resolve(i) of Algorithm 1: empty S_i if it holds anything, then fill B_i
// if it is below capacity and a deeper level holds anything.
template <class Team>
__device__ void resolve(Team &t, Smem &S, int i)
{
    if (S.hs.L[i].slen > 0) {
        PhaseTimer<Team> pt(t, i == 0 ? STAT_T_EMPTY : STAT_T_DEEP);
        empty_level(t, S, i);
    }
    resolve_fill(t, S, i);
}

// The rest of Resolve(i) once S_i is empty: Fill(B_i) if B_i is below
// capacity and a deeper level holds anything; count the Resolve.
template <class Team>
__device__ void resolve_fill(Team &t, Smem &S, int i)
{
    if (t.failed()) return;
    if (i + 1 < (int)S.hs.q && S.hs.L[i].blen < S.hs.L[i].capB && deeper_nonempty(S.hs, i)) {
        PhaseTimer<Team> pt(t, i == 0 ? STAT_T_FILL : STAT_T_DEEP);
        fill_level(t, S, i);
    }
    LEADER
    {
        S.hs.L[i].nres++;
        if (t.cta() == 0) stat_add(t.sc.stats + STAT_RES0 + i, 1);
    }
    __syncthreads();
}

// The schedule after every operation (Theorem 3): Resolve(0), and Resolve(i)
// after every fourth Resolve(i-1).  With `emptied`, Empty(S_0) of this
// Resolve(0) already ran (fused with the batch sort).
template <class Team>
__device__ void resolve_schedule(Team &t, Smem &S, bool emptied = false)
{
    if (emptied) {
        for (int j = 1; j < (int)S.hs.q && !t.failed(); j++) { // Empty's cascade
            if (S.hs.L[j].slen <= S.hs.L[j].capS) break;
            empty_level_once(t, S, j);
        }
        resolve_fill(t, S, 0);
    } else {
        resolve(t, S, 0);
    }
    for (int i = 1; i < (int)S.hs.q && !t.failed(); i++) {
        if (S.hs.L[i - 1].nres % 4 != 0) break;
        resolve(t, S, i);
    }
}

// Guarantee before an extract of r: B_0 holds at least r elements, or every
// live element.  Stale drops can leave B_0 short of Theorem 3's counts; then
// all signal buffers are emptied top-down and all buckets filled bottom-up
// (the sequential bucket heap's Fill cascade, Section 2.1).
template <class Team>
__device__ void ensure_top(Team &t, Smem &S, u64 r)
{
    if (S.hs.L[0].blen >= r || !deeper_nonempty(S.hs, 0)) return;
    PhaseTimer<Team> pt(t, STAT_T_ENSURE);
    for (int i = 0; i < (int)S.hs.q && !t.failed(); i++)
        if (S.hs.L[i].slen > 0) empty_level_once(t, S, i);
    for (int i = (int)S.hs.q - 2; i >= 0 && !t.failed(); i--)
        if (S.hs.L[i].blen < S.hs.L[i].capB && deeper_nonempty(S.hs, i)) fill_level(t, S, i);
}

// Sort the BulkUpdate elements staged in U[src][0, n) into S_0.  n <= d.
template <class Team>
__device__ void bulk_sort(Team &t, Smem &S, u64 n, int src = 0)
{
    HeapState &hs = S.hs;
    if (n > 0) {
        u64 *sorted;
        {
            PhaseTimer<Team> pt(t, STAT_T_SORT);
            // SSSP stages vertex ids; their final packed distances are gathered here
            const u64 *gather = hs.mark ? hs.cur : nullptr;
            // small batches: rank sort across the team (one barrier); the
            // quadratic count only pays while the team has many warps (one
            // CTA sorts faster with the block sort at every batch size)
            if (!Team::kSingle && n <= TILE) {
                team_rank_sort(t, S, hs.U[src], (u32)n, hs.U[src ^ 1], gather);
                sorted = hs.U[src ^ 1];
            } else {
                sorted = team_sort(t, S, hs.U[src], n, hs.U[src ^ 1], gather);
            }
        }
        LEADER
        {
            hs.L[0].ssel = (sorted == hs.U[0]) ? 0 : 1;
            hs.L[0].shead = 0;
            hs.L[0].slen = n;
            if (t.cta() == 0) *t.sc.ucount = 0;
        }
        __syncthreads();
    }
}

// After the BulkUpdate elements were staged in U[src][0, n): sort them into
// S_0, then Resolve(0) and the schedule.  n <= d.
template <class Team>
__device__ void bulk_commit(Team &t, Smem &S, u64 n, int src = 0)
{
    bulk_sort(t, S, n, src);
    resolve_schedule(t, S);
}

// The BulkUpdate of an SSSP round: the staged vertex ids (one per key, each
// its final word) are sorted into S_0 and Resolve(0) runs; with a multi-CTA
// team and a small batch the sort is fused with Empty(S_0).  Returns the
// batch size.  With take > 0, when the round's bookkeeping takes the single
// step (nothing below level 0), the next round's extract of up to take
// words is applied too and *taken receives its size (else *taken stays
// unchanged).
// Per-query counters kept in registers and added to the statistics once per
// query (a reduction per round on the critical path cost about 0.15 us per
// round): the single-step commit's, by CTA 0's thread 0, and each CTA's
// scanned arcs, by its thread 0.
struct RoundCounts {
    u64 stale = 0, merged = 0, res0 = 0, improve = 0;
    u64 relaxed = 0; // arcs this CTA scanned (every CTA's thread 0 adds its own)
};

template <class Team>
__device__ u64 sssp_commit(Team &t, Smem &S, u64 take = 0, u64 *taken = nullptr, RoundCounts *rc = nullptr)
{
    if constexpr (!Team::kSingle) {
        HeapState &hs = S.hs;
        Level &L = hs.L[0];
        const u64 per = (L.blen + t.ncta() - 1) / t.ncta();
        if (per <= TILE && L.slen == 0) {
            u64 n = 0;
            int how;
            bool done = false;
            {
                PhaseTimer<Team> pt(t, STAT_T_EMPTY);
                u64 total = 0;
                const u64 nb = L.blen;
                how = empty0_fused(t, S, &n, &total);
                if (how == FUSED_OK && !t.failed()) {
                    if (L.T == INF && total <= L.capB && !deeper_nonempty(hs, 0)) {
                        // Empty keeps the whole merged run in B_0 and no level
                        // below 0 holds anything: this Resolve(0) and every
                        // Resolve(i) the Theorem 3 schedule runs now only
                        // count themselves (uniform: every CTA summed the
                        // same partials)
                        // with take, the next round's extract too: the
                        // first min(take, total) words of the new B_0
                        const u64 nf = take < total ? take : total;
                        LEADER
                        {
                            L.bsel ^= 1;
                            L.bhead = nf;
                            L.blen = total - nf;
                            L.slen = 0;
                            L.shead = 0;
                            const bool own = t.cta() == 0 && rc;
                            if (own) {
                                rc->stale += n + nb - total;
                                rc->merged += n + nb;
                                rc->res0++;
                            } else if (t.cta() == 0) {
                                stat_add(t.sc.stats + STAT_STALE, n + nb - total);
                                stat_add(t.sc.stats + STAT_MERGED, n + nb);
                                stat_add(t.sc.stats + STAT_RES0, 1);
                            }
                            hs.L[0].nres++;
                            for (int i = 1; i < (int)hs.q; i++) {
                                if (hs.L[i - 1].nres % 4 != 0) break;
                                hs.L[i].nres++;
                                if (t.cta() == 0) stat_add(t.sc.stats + STAT_RES0 + i, 1);
                            }
                        }
                        __syncthreads();
                        done = true;
                        if (taken && take) *taken = nf;
                    } else {
                        empty_split(t, S, 0, L.B[L.bsel ^ 1], n, L.blen, total);
                    }
                }
            }
            if (how == FUSED_OK) {
                if (!done && !t.failed()) resolve_schedule(t, S, true);
                return n;
            }
            if (how == FUSED_NO) bulk_commit(t, S, n);
            return n;
        }
    }
    const u64 n = ldg_cg(t.sc.ucount);
    bulk_commit(t, S, n);
    return n;
}

// Load / store the replicated control state.
__device__ __forceinline__ void state_load(Smem &S, const HeapState *g)
{
    const u64 *src = reinterpret_cast<const u64 *>(g);
    u64 *dst = reinterpret_cast<u64 *>(&S.hs);
    for (u32 i = threadIdx.x; i < sizeof(HeapState) / 8; i += NT) dst[i] = ldg_cg(src + i);
    __syncthreads();
}

__device__ __forceinline__ void state_store(const Smem &S, HeapState *g)
{
    const u64 *src = reinterpret_cast<const u64 *>(&S.hs);
    u64 *dst = reinterpret_cast<u64 *>(g);
    for (u32 i = threadIdx.x; i < sizeof(HeapState) / 8; i += NT) dst[i] = src[i];
}

static_assert(sizeof(HeapState) % 8 == 0, "state is copied as words");

// ---------------------------------------------------------- parDijkstra

struct Graph {
    u32 n;
    u64 m;
    const u64 *row_ptr;
    const u32 *col;
    const u32 *w;
};

// Append the improved words of this pass to U (block-aggregated: one global
// atomic per CTA pass).  All threads of the CTA call it.
__device__ __forceinline__ void block_emit(bool imp, u64 P, u64 *U, u64 ucap, u64 *ucount, u32 *err, Smem &S)
{
    u32 tot;
    const u32 excl = block_scan(imp ? 1u : 0u, &tot, S);
    if (tot == 0) return;
    if (threadIdx.x == 0) S.bc[7] = atomicAdd(ucount, (u64)tot);
    __syncthreads();
    const u64 base = S.bc[7];
    if (imp) {
        const u64 pos = base + excl;
        if (pos < ucap)
            U[pos] = P;
        else
            raise_err(err, ST_CAPACITY, 6);
    }
    __syncthreads();
}

// Append each thread's improved words (up to 4) to U, one global atomic per
// CTA pass.  All threads of the CTA call it.
template <int RA>
__device__ __forceinline__ void block_emit_n(u32 nimp, const u64 (&Pw)[RA], const bool (&act)[RA], u64 *U, u64 ucap,
                                             u64 *ucount, u32 *err, Smem &S)
{
    u32 tot;
    const u32 excl = block_scan(nimp, &tot, S);
    if (tot == 0) return;
    if (threadIdx.x == 0) S.bc[7] = atomicAdd(ucount, (u64)tot);
    __syncthreads();
    u64 pos = S.bc[7] + excl;
#pragma unroll
    for (int k = 0; k < RA; k++) {
        if (act[k]) {
            if (pos < ucap)
                U[pos] = Pw[k];
            else
                raise_err(err, ST_CAPACITY, 6);
            pos++;
        }
    }
    __syncthreads();
}

// Relax every out-arc of the frontier F[0, nf) (packed (dist << kb) | u
// words): nd = dist(u) + w; atomicMin on the packed tentative distance of v;
// improved words go to U for the BulkUpdate (Section 4.1, steps 2-3).
// Returns the arcs this CTA scanned (the caller adds them to the statistics
// once per query).  Frontiers of up to FMAX vertices are split by arcs over the team (every
// CTA computes the degree prefix itself); larger ones by vertices.
template <class Team>
__device__ u64 relax(Team &t, Smem &S, const Graph &g, u64 *Dist, const u64 *F, u32 nf, u32 kb, u64 dmax,
                      u64 *U, u64 ucap, u32 *mark, u32 tag, u64 maxdeg)
{
    constexpr int RA = 4; // arcs per thread per pass, loads issued together (memory-level parallelism)
    const u32 tid = threadIdx.x;
    const u64 vmask = (kb >= 64) ? INF : ((1ull << kb) - 1);
    u64 *rb = S.win;                                   // row begin of staged frontier vertices
    u64 *du = S.win + FMAX;                            // their distances
    u32 *off = reinterpret_cast<u32 *>(S.keep + FMAX / 2); // degree prefix (FMAX + 1 entries)
#ifdef PBH_BULK_RELAX
    constexpr u32 BULK_ARCS = 1024;                                    // arcs staged per chunk
    u32 *bulk_col = reinterpret_cast<u32 *>(S.keep + FMAX + 8);        // staged col rows (16-byte aligned)
    u32 *bulk_w = reinterpret_cast<u32 *>(S.keep + FMAX + 8 + BULK_ARCS / 2); // staged w rows
    static_assert(FMAX + 8 + BULK_ARCS <= TILE + 8, "staging slots must fit in keep");
#endif
    const u64 P = t.ncta(), c = t.cta();
    // Split by vertices when every CTA's share of the frontier has at most
    // one pass of arcs (NT * RA): each CTA then reads only its own frontier
    // words and row pointers, not the whole frontier.  Otherwise small
    // frontiers of high-degree vertices are split by arcs (every CTA computes
    // the degree prefix of the whole frontier), and frontiers of more than
    // FMAX vertices by vertices, in chunks of FMAX.
    const bool one_pass = ((u64)nf + P - 1) / P * maxdeg <= (u64)NT * RA;
    const bool by_arcs = nf <= (u32)FMAX && !one_pass;
    u64 v0, v1;
    if (by_arcs) {
        v0 = 0;
        v1 = nf;
    } else {
        v0 = (u64)nf * c / P;
        v1 = (u64)nf * (c + 1) / P;
    }
    u64 relaxed_local = 0;
    for (u64 cb = v0; cb < v1; cb += FMAX) {
        const u32 cn = (u32)min((u64)FMAX, v1 - cb);
        // stage the chunk: row begins, distances, degrees (4 vertices per thread)
        constexpr int FV = FMAX / NT; // frontier vertices per thread
        u32 dg[FV];
        u64 xs[FV], bs[FV], es[FV];
        u32 sum = 0;
#pragma unroll
        for (int k = 0; k < FV; k++) {
            const u32 j = tid * FV + k;
            xs[k] = j < cn ? ldg_cg(F + cb + j) : 0;
        }
#pragma unroll
        for (int k = 0; k < FV; k++) {
            const u32 j = tid * FV + k;
            const u64 u = xs[k] & vmask;
            bs[k] = es[k] = 0;
            if (j < cn && u < g.n) {
                bs[k] = __ldg(g.row_ptr + u);
                es[k] = __ldg(g.row_ptr + u + 1);
            } else if (j < cn) {
                raise_err(t.sc.err, ST_CAPACITY, 24);
            }
        }
#pragma unroll
        for (int k = 0; k < FV; k++) {
            const u32 j = tid * FV + k;
            dg[k] = 0;
            if (j < cn) {
                rb[j] = bs[k];
                du[j] = xs[k] >> kb;
                dg[k] = (es[k] >= bs[k] && es[k] <= g.m) ? (u32)(es[k] - bs[k]) : 0;
            }
            sum += dg[k];
        }
#ifdef PBH_BULK_RELAX
        // Stage the arc rows of this chunk's vertices into shared memory with
        // one bulk copy per row and array (col, w), into fixed slots of
        // slot_w words per vertex, so the copies are in flight during the
        // degree prefix below.  Rows that do not start and end on a 16-byte
        // boundary keep plain loads (flag bit 31 of their row begin).
        const u32 slot_w = (u32)((maxdeg + 3) & ~3ull);
        const bool bulk = !by_arcs && one_pass && (u64)cn * slot_w <= BULK_ARCS;
        if (bulk) {
            u32 bytes = 0;
#pragma unroll
            for (int k = 0; k < FV; k++) {
                const u32 j = tid * FV + k;
                if (j < cn && dg[k] > 0 && (bs[k] & 3) == 0 && (dg[k] & 3) == 0) {
                    bulk_g2s(bulk_col + j * slot_w, g.col + bs[k], 4 * dg[k], &S.mbar);
                    bulk_g2s(bulk_w + j * slot_w, g.w + bs[k], 4 * dg[k], &S.mbar);
                    bytes += 8 * dg[k];
                } else if (j < cn) {
                    rb[j] |= 1ull << 63; // this row is read with plain loads
                }
            }
            sum |= bytes << 13; // bytes / 8 <= BULK_ARCS fits beside the degree sum (< 2^13 here)
            if (tid == 0) S.mbar_late = 0; // ordered before the wait by the scan's barriers
        }
#endif
        u32 total;
        u32 excl = block_scan(sum, &total, S);
#ifdef PBH_BULK_RELAX
        if (bulk) {
            const u32 bytes = total >> 13;
            total &= (1u << 13) - 1;
            excl &= (1u << 13) - 1;
            if (tid == 0) mbar_arrive_expect(&S.mbar, bytes);
        }
#endif
#pragma unroll
        for (int k = 0; k < FV; k++) {
            const u32 j = tid * FV + k;
            if (j < cn) off[j] = excl;
            excl += dg[k];
        }
        if (tid == 0) off[cn] = total;
        __syncthreads();
#ifdef PBH_BULK_RELAX
        bool staged = false;
        if (bulk) {
            const u32 ph = S.mbar_phase;
            if (!mbar_wait(&S.mbar, ph)) S.mbar_late = 1;
            __syncthreads();
            staged = S.mbar_late == 0; // uniform: the copies did not land in time means never read the slots
            if (tid == 0) {
                S.mbar_phase = ph ^ 1;
                if (!staged) raise_err(t.sc.err, ST_TIMEOUT, 27);
            }
        }
#endif
        PBH_PROBE(t, 1); // frontier words, row pointers, degree prefix
        u64 e0, e1;
        if (by_arcs) {
            e0 = (u64)total * c / P;
            e1 = (u64)total * (c + 1) / P;
        } else {
            e0 = 0;
            e1 = total;
        }
        relaxed_local += e1 - e0;
        for (u64 eb = e0; eb < e1; eb += (u64)NT * RA) {
            u64 idx[RA], dd[RA];
            bool act[RA];
#pragma unroll
            for (int k = 0; k < RA; k++) {
                const u64 e = eb + (u64)k * NT + tid;
                act[k] = e < e1;
                idx[k] = 0;
                dd[k] = 0;
                if (act[k]) {
                    u32 lo = 0, hi = cn; // last j with off[j] <= e
                    while (hi - lo > 1) {
                        const u32 mid = (lo + hi) >> 1;
                        if (off[mid] <= e)
                            lo = mid;
                        else
                            hi = mid;
                    }
#ifdef PBH_BULK_RELAX
                    if (staged && !(rb[lo] >> 63)) {
                        idx[k] = (1ull << 63) | ((u64)lo * slot_w + (e - off[lo])); // a slot in shared memory
                    } else
#endif
                        idx[k] = (rb[lo] & ~(1ull << 63)) + (e - off[lo]);
                    dd[k] = du[lo];
                }
            }
            u32 vv[RA], ww[RA];
#pragma unroll
            for (int k = 0; k < RA; k++) {
#ifdef PBH_BULK_RELAX
                if (act[k] && (idx[k] >> 63)) {
                    const u32 sidx = (u32)idx[k];
                    vv[k] = bulk_col[sidx];
                    ww[k] = bulk_w[sidx];
                    continue;
                }
#endif
                if (act[k] && idx[k] >= g.m) {
                    raise_err(t.sc.err, ST_CAPACITY, 22);
                    act[k] = false;
                }
                vv[k] = act[k] ? __ldg(g.col + idx[k]) : 0;
                ww[k] = act[k] ? __ldg(g.w + idx[k]) : 0;
            }
            u64 Pw[RA], old[RA];
#pragma unroll
            for (int k = 0; k < RA; k++) {
                Pw[k] = 0;
                old[k] = 0;
                if (!act[k]) continue;
                const u64 nd = dd[k] + ww[k];
                if (vv[k] >= g.n) {
                    raise_err(t.sc.err, ST_INVAL, 7); // arc target outside the graph
                    act[k] = false;
                } else if (nd > dmax) {
                    raise_err(t.sc.err, ST_RANGE, 8);
                    act[k] = false;
                } else {
                    Pw[k] = (nd << kb) | vv[k];
                    old[k] = atomicMin(Dist + vv[k], Pw[k]);
                }
            }
            // stage each improved vertex once per round: the first thread whose
            // atomicMin lowered it claims it (the batch keeps one word per key,
            // its final minimum, gathered at sort time)
            u32 nimp = 0;
#pragma unroll
            for (int k = 0; k < RA; k++) {
                if (act[k] && old[k] > Pw[k] && atomicExch(mark + vv[k], tag) != tag) {
                    Pw[k] = vv[k];
                    nimp++;
                } else {
                    act[k] = false;
                }
            }
            PBH_PROBE(t, 2); // arc loads, atomicMin, claims
            block_emit_n(nimp, Pw, act, U, ucap, t.sc.ucount, t.sc.err, S);
            PBH_PROBE(t, 3); // staging (block scan, slot reservation, stores)
        }
        __syncthreads();
    }
    return relaxed_local;
}

// Largest out-degree (team reduction into stats[STAT_MAXDEG]).  Ends with a barrier.
template <class Team>
__device__ u64 team_max_degree(Team &t, Smem &S, const Graph &g)
{
    u64 mx = 0;
    const u64 stride = (u64)t.ncta() * NT;
    for (u64 v = (u64)t.cta() * NT + threadIdx.x; v < g.n; v += stride) {
        const u64 dgv = __ldg(g.row_ptr + v + 1) - __ldg(g.row_ptr + v);
        mx = dgv > mx ? dgv : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const u64 y = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = y > mx ? y : mx;
    }
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(t.sc.stats + STAT_MAXDEG, mx);
    t.sync();
    return ldg_cg(t.sc.stats + STAT_MAXDEG);
}

// Smallest arc weight (team reduction into stats[STAT_WMIN], which holds
// the bitwise complement so that a zeroed header reads as "no arc yet").
// Ends with a barrier.
template <class Team>
__device__ u64 team_min_weight(Team &t, Smem &S, const Graph &g)
{
    u64 mn = 0xffffffffull;
    const u64 stride = (u64)t.ncta() * NT;
    for (u64 e = (u64)t.cta() * NT + threadIdx.x; e < g.m; e += stride) {
        const u64 w = __ldg(g.w + e);
        mn = w < mn ? w : mn;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const u64 y = __shfl_xor_sync(0xffffffffu, mn, o);
        mn = y < mn ? y : mn;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(t.sc.stats + STAT_WMIN, ~mn);
    t.sync();
    const u64 v = ~ldg_cg(t.sc.stats + STAT_WMIN);
    return v > 0xffffffffull ? 0xffffffffull : v; // no arcs: any bound works
}

// A whole parDijkstra query run by one team.  S.hs holds the empty heap laid
// out for this query (cur = Dist).  Dist: n words, receives distances.
template <class Team>
__device__ void run_query(Team &t, Smem &S, const Graph &g, u32 source, u64 *Dist, u32 r, u32 kb, u64 limit_ns)
{
    HeapState &hs = S.hs;
    const u64 stride = (u64)t.ncta() * NT;
    const u64 gtid = (u64)t.cta() * NT + threadIdx.x;
    const u64 dmax = (kb >= 64) ? 0 : ((INF >> kb) - 1); // largest distance that packs (INF stays reserved)
    t.init();
#ifdef PBH_BULK_RELAX
    if (threadIdx.x == 0) {
        mbar_init(&S.mbar);
        S.mbar_phase = 0;
    }
    __syncthreads();
#endif
    if constexpr (Team::kSoftBarrier) {
        // the stall test: CTA 0 withholds its arrival at the next barrier (the
        // one after the degree pass), so every CTA's bounded wait expires; all
        // CTAs have finished the work before it, so nothing reads unready data
        if (t.sc.stall && t.cta() == 0 && threadIdx.x == 0) t.withhold = true;
    }
    for (u64 v = gtid; v < g.n; v += stride) {
        Dist[v] = INF;
        hs.mark[v] = 0;
    }
    const u64 maxdeg = team_max_degree(t, S, g);
    // settle criterion (Section 1's Dijkstra invariant, as in Crauser et
    // al.'s OUT criterion with one global bound): every heap vertex whose
    // tentative distance is at most min + w_min is final, since any other
    // path reaches it through a heap vertex and at least one more arc
    const u64 wmin = hs.settle ? team_min_weight(t, S, g) : 0;
    const u64 r_cap = maxdeg ? hs.d / maxdeg : hs.d; // widest frontier whose lowerings fit a batch of d
    u64 settled = 0;
    u64 r_eff = maxdeg ? hs.d / maxdeg : hs.d;
    if (r_eff > r) r_eff = r;
    if (maxdeg > hs.d || r_eff == 0) raise_err(t.sc.err, ST_INVAL, 9);
    if (gtid == 0) {
        const u64 ps = (u64)source; // distance 0
        Dist[source] = ps;
        hs.U[0][0] = source;       // staged as a vertex id, like every SSSP BulkUpdate element
        *t.sc.ucount = 1;
        t.sc.stats[STAT_REFF] = r_eff;
        t.sc.stats[STAT_LEVELS] = hs.q;
    }
    t.sync();
    if (t.failed()) return;
    sssp_commit(t, S); // the source
    PBH_PROBE_START(t);
    u64 rounds = 0, extracted = 0;
    // Liveness bounds: every round extracts at least one element and an
    // element re-enters only when a distance strictly falls, so a correct run
    // ends long before either bound; they only turn a defect into an error.
    const u64 max_rounds = 64ull * g.n + 1024;
    const u64 limit = limit_ns ? limit_ns : QUERY_NS + QUERY_NS_PER_VERTEX * (u64)g.n;
    const u64 t_start = gtimer();
    u64 pre = ~0ull; // the size of a frontier the commit already took (~0: none)
    RoundCounts counts; // added to the statistics at the end (thread 0)
    while (!t.failed()) {
        Level &L0 = hs.L[0];
        u64 nf;
        const u64 *F;
        if (pre != ~0ull) {
            nf = pre;
            if (nf == 0) break;
            F = L0.B[L0.bsel] + L0.bhead - nf;
        } else {
            ensure_top(t, S, r_eff);
            if (t.failed()) break;
            nf = L0.blen < r_eff ? L0.blen : r_eff;
            if (nf == 0) break;
            F = L0.B[L0.bsel] + L0.bhead;
            if (hs.settle && nf < r_cap && nf < L0.blen) {
                // B_0 starts with the heap minimum; take every word of B_0 whose
                // distance is at most min + w_min as well (up to r_cap)
                const u64 dmin = team_load<Team>(S, F) >> kb;
                if (dmin + wmin < dmax) {
                    const u64 last = ((dmin + wmin + 1) << kb) - 1; // largest word of distance min + w_min
                    u64 ns = team_count_le(t, S, F, L0.blen, last);
                    if (ns > r_cap) ns = r_cap;
                    if (ns > nf) {
                        settled += ns - nf;
                        nf = ns;
                    }
                }
            }
            __syncthreads();
            LEADER
            {
                L0.bhead += nf;
                L0.blen -= nf;
            }
            __syncthreads();
        }
        PBH_PROBE(t, 0); // loop control, ensure_top, extraction
        PBH_SPAN_BEGIN();
        {
            PhaseTimer<Team> pt(t, STAT_T_RELAX);
            counts.relaxed +=
                relax(t, S, g, Dist, F, (u32)nf, kb, dmax, hs.U[0], hs.d, hs.mark, (u32)rounds + 1, maxdeg);
            if (t.cta() == 0 && threadIdx.x == 0 && (rounds > max_rounds || gtimer() - t_start > limit))
                raise_err(t.sc.err, ST_TIMEOUT, 10); // seen by every CTA after the barrier below
            PBH_SPAN_END(t, 14); // relax, per CTA (sum, max)
            t.sync();
            PBH_PROBE(t, 4); // relax barrier
            PBH_SPAN_BEGIN();
        }
        if (t.failed()) break;
        pre = ~0ull;
        const u64 nu = sssp_commit(t, S, hs.settle ? 0 : r_eff, &pre, &counts);
        PBH_PROBE(t, 13); // Empty's split, the Theorem 3 schedule
        rounds++;
        extracted += nf;
        counts.improve += nu;
    }
    if (threadIdx.x == 0 && counts.relaxed) stat_add(t.sc.stats + STAT_RELAX, counts.relaxed);
    if (t.cta() == 0 && threadIdx.x == 0) {
        stat_add(t.sc.stats + STAT_IMPROVE, counts.improve);
        stat_add(t.sc.stats + STAT_STALE, counts.stale);
        stat_add(t.sc.stats + STAT_MERGED, counts.merged);
        stat_add(t.sc.stats + STAT_RES0, counts.res0);
        t.sc.stats[STAT_ROUNDS] = rounds;
        t.sc.stats[STAT_EXTRACTED] = extracted;
        t.sc.stats[STAT_SETTLED] = settled;
        t.sc.stats[STAT_SYNCS] = t.nsync;
    }
    t.sync();
    for (u64 v = gtid; v < g.n; v += stride) {
        const u64 x = ldg_cg(Dist + v);
        Dist[v] = x == INF ? INF : (x >> kb);
    }
}

} // namespace pbhk
