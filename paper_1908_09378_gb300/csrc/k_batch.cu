// k_batch.cu -- many independent parDijkstra queries in one persistent
// launch: each CTA takes queries from a device work queue and runs each with
// its own heap (CtaTeam).
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

} // namespace

namespace pbhk {
const void *kfn_sssp_batch() { return reinterpret_cast<const void *>(&k_sssp_batch); }
} // namespace pbhk
