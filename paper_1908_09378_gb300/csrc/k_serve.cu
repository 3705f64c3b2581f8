// k_serve.cu -- the continuous-batching server: one persistent launch whose
// CTAs (or thread-block clusters) take queries from a request ring in
// pinned, device-mapped host memory.
//
// Device code: core.cuh.  Host ABI: pbh.cu.
#include "kernels.h"

using namespace pbhk;

namespace {

__device__ __forceinline__ Smem &smem()
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    return *reinterpret_cast<Smem *>(smem_raw);
}

// ------------------------------------------------------------ serving
//
// A persistent kernel whose CTAs take requests from a ring that the host
// writes into pinned, device-mapped memory.  Request k goes to slot
// k % slots; the host publishes it by advancing ctl->tail and may reuse the
// slot once done[slot] reports k + 1.  Each CTA claims the next request
// number, waits (bounded) until it is published, runs the query with its own
// heap (CtaTeam) and writes its completion flag and device timestamps.

__global__ void __launch_bounds__(NT) k_serve(const ServeRecord *ring, ServeCtl *ctl, u64 *done, u64 *t_begin,
                                             u64 *t_end, u32 slots, u64 *head)
{
    Smem &S = smem();
    for (;;) {
        if (threadIdx.x == 0) {
            const u64 idx = atomicAdd(head, 1ull);
            u64 ok = 1;
            // the wait is bounded by the host's silence: it restarts whenever
            // the host publishes a request or advances its heartbeat
            u64 t0 = gtimer(), seen = 0;
            for (u32 spin = 0; *(volatile u64 *)&ctl->tail <= idx; spin++) {
                if (*(volatile u32 *)&ctl->stop) {
                    ok = 0;
                    break;
                }
                if ((spin & 63) == 0) {
                    const u64 now = gtimer();
                    const u64 sign = *(volatile u64 *)&ctl->heartbeat + *(volatile u64 *)&ctl->tail;
                    if (sign != seen) {
                        seen = sign;
                        t0 = now;
                    }
                    const u64 idle_set = *(volatile u64 *)&ctl->idle_ns;
                    if (now - t0 > (idle_set ? idle_set : SERVE_IDLE_NS)) {
                        atomicCAS(&ctl->status, 0u, (u32)ST_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(1000);
            }
            __threadfence_system(); // acquire the published record
            S.bc[0] = idx;
            S.bc[1] = ok;
        }
        __syncthreads();
        const u64 idx = S.bc[0];
        const bool ok = S.bc[1] != 0;
        __syncthreads();
        if (!ok) break;
        const u32 slot = (u32)(idx % slots);
        const ServeRecord &rec = ring[slot];
        const QueryDesc q = rec.q; // one copy out of host memory
        if (threadIdx.x == 0) t_begin[slot] = gtimer();
        for (u64 i = threadIdx.x; i < q.header_words; i += NT) q.header[i] = 0;
        if (threadIdx.x == 0) g_err_sink_set(q.sc.err);
        __syncthreads();
        state_load(S, q.hs);
        CtaTeam t{q.sc};
        run_query(t, S, q.g, q.source, q.dist, q.r, q.kb, q.limit_ns);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence_system(); // results before the flag
            t_end[slot] = gtimer();
            *(volatile u64 *)&done[slot] = idx + 1;
        }
    }
}

// The same server with one thread-block cluster per request (ClusterTeam):
// for large queries, whose one-CTA run would set the latency tail.  The
// cluster's first CTA claims and waits for the request; the others read the
// claim from its shared memory.
__global__ void __launch_bounds__(NT, 1) k_serve_cluster(const ServeRecord *ring, ServeCtl *ctl, u64 *done,
                                                        u64 *t_begin, u64 *t_end, u32 slots, u64 *head)
{
    Smem &S = smem();
    const u32 rank = cluster_rank();
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) {
            const u64 idx = atomicAdd(head, 1ull);
            u64 ok = 1;
            // the wait is bounded by the host's silence: it restarts whenever
            // the host publishes a request or advances its heartbeat
            u64 t0 = gtimer(), seen = 0;
            for (u32 spin = 0; *(volatile u64 *)&ctl->tail <= idx; spin++) {
                if (*(volatile u32 *)&ctl->stop) {
                    ok = 0;
                    break;
                }
                if ((spin & 63) == 0) {
                    const u64 now = gtimer();
                    const u64 sign = *(volatile u64 *)&ctl->heartbeat + *(volatile u64 *)&ctl->tail;
                    if (sign != seen) {
                        seen = sign;
                        t0 = now;
                    }
                    const u64 idle_set = *(volatile u64 *)&ctl->idle_ns;
                    if (now - t0 > (idle_set ? idle_set : SERVE_IDLE_NS)) {
                        atomicCAS(&ctl->status, 0u, (u32)ST_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
                __nanosleep(1000);
            }
            __threadfence_system(); // acquire the published record
            S.bc[0] = idx;
            S.bc[1] = ok;
        }
        cluster_barrier();
        const u64 idx = rank == 0 ? S.bc[0] : dsmem_ld_u64(&S.bc[0], 0);
        const bool ok = (rank == 0 ? S.bc[1] : dsmem_ld_u64(&S.bc[1], 0)) != 0;
        cluster_barrier(); // every CTA has read the claim before the next one
        if (!ok) break;
        const u32 slot = (u32)(idx % slots);
        const QueryDesc q = ring[slot].q; // one copy out of host memory per CTA
        if (rank == 0) {
            if (threadIdx.x == 0) t_begin[slot] = gtimer();
            for (u64 i = threadIdx.x; i < q.header_words; i += NT) q.header[i] = 0;
        }
        if (threadIdx.x == 0) g_err_sink_set(q.sc.err);
        cluster_barrier(); // the cleared header before any CTA of the query starts
        state_load(S, q.hs);
        ClusterTeam t{q.sc};
        run_query(t, S, q.g, q.source, q.dist, q.r, q.kb, q.limit_ns);
        cluster_barrier(); // every CTA's results before the completion flag
        if (rank == 0 && threadIdx.x == 0) {
            __threadfence_system(); // results before the flag
            t_end[slot] = gtimer();
            *(volatile u64 *)&done[slot] = idx + 1;
        }
    }
}

} // namespace

namespace pbhk {
const void *kfn_serve() { return reinterpret_cast<const void *>(&k_serve); }
const void *kfn_serve_cluster() { return reinterpret_cast<const void *>(&k_serve_cluster); }
} // namespace pbhk
