// k_grid.cu -- one parDijkstra query on the whole GPU: a cooperative grid of
// one CTA per SM (GridTeam) runs every round of Section 4.1 inside the launch.
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

// Copy the HeapState kernel argument into shared memory (every CTA).
__device__ __forceinline__ void state_from_param(Smem &S, const HeapState &p)
{
    const u64 *src = reinterpret_cast<const u64 *>(&p);
    u64 *dst = reinterpret_cast<u64 *>(&S.hs);
    for (u32 i = threadIdx.x; i < sizeof(HeapState) / 8; i += NT) dst[i] = src[i];
    __syncthreads();
}

__global__ void __launch_bounds__(NT, 1) k_sssp_grid(Scratch sc, HeapState hs0, Graph g, u32 source, u64 *dist, u32 r,
                                                   u32 kb, u64 limit_ns)
{
    Smem &S = smem();
    state_from_param(S, hs0);
    GridQueryTeam t{sc};
    if (threadIdx.x == 0) g_err_sink_set(sc.err, sc.bar);
    run_query(t, S, g, source, dist, r, kb, limit_ns);
}

} // namespace

namespace pbhk {
const void *kfn_sssp_grid() { return reinterpret_cast<const void *>(&k_sssp_grid); }
} // namespace pbhk
