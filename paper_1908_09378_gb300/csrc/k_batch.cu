// k_batch.cu -- many independent parDijkstra queries in one persistent
// launch: each CTA takes queries from a device work queue and runs each with
// its own heap (CtaTeam); the largest queries of a batch can run instead on
// thread-block clusters (ClusterTeam), in a second launch beside the first.
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

__global__ void __launch_bounds__(NT) k_sssp_batch(const QueryDesc *qs, const u32 *order, u32 nq, u32 *next)
{
    Smem &S = smem();
    for (;;) {
        if (threadIdx.x == 0) S.bc[0] = atomicAdd(next, 1u);
        __syncthreads();
        const u32 qi = (u32)S.bc[0];
        __syncthreads();
        if (qi >= nq) break;
        const QueryDesc &q = qs[order[qi]];
        for (u64 i = threadIdx.x; i < q.header_words; i += NT) q.header[i] = 0;
        if (threadIdx.x == 0) g_err_sink_set(q.sc.err);
        __syncthreads();
        state_load(S, q.hs);
        CtaTeam t{q.sc};
        const Graph g = q.g;
        run_query(t, S, g, q.source, q.dist, q.r, q.kb, q.limit_ns);
        __syncthreads();
    }
}

// The large queries of a batch, each on one thread-block cluster
// (ClusterTeam): the first CTA of a cluster claims the next query, the others
// read its number from that CTA's shared memory.
__global__ void __launch_bounds__(NT, 1) k_sssp_batch_cluster(const QueryDesc *qs, const u32 *order, u32 nq, u32 *next)
{
    Smem &S = smem();
    const u32 rank = cluster_rank();
    for (;;) {
        if (rank == 0 && threadIdx.x == 0) S.bc[0] = atomicAdd(next, 1u);
        cluster_barrier();
        const u32 qi = (u32)(rank == 0 ? S.bc[0] : dsmem_ld_u64(&S.bc[0], 0));
        cluster_barrier(); // every CTA has read the number before the next claim
        if (qi >= nq) break;
        const QueryDesc &q = qs[order[qi]];
        if (rank == 0)
            for (u64 i = threadIdx.x; i < q.header_words; i += NT) q.header[i] = 0;
        if (threadIdx.x == 0) g_err_sink_set(q.sc.err);
        cluster_barrier(); // the cleared header before any CTA of the query starts
        state_load(S, q.hs);
        ClusterTeam t{q.sc};
        const Graph g = q.g;
        run_query(t, S, g, q.source, q.dist, q.r, q.kb, q.limit_ns);
        cluster_barrier();
    }
}

} // namespace

namespace pbhk {
const void *kfn_sssp_batch() { return reinterpret_cast<const void *>(&k_sssp_batch); }
const void *kfn_sssp_batch_cluster() { return reinterpret_cast<const void *>(&k_sssp_batch_cluster); }
} // namespace pbhk
