// k_op.cu -- the heap-API kernels: one heap operation per cooperative launch
// (BulkUpdate, assign, delete or extract, then Resolve(0) and the Theorem 3
// schedule), the debug validator, and a fill helper.
//
// Device code: heapop.cuh, core.cuh.  Host ABI: pbh.cu.
#include "kernels.h"
#include "heapop.cuh"

using namespace pbhk;

namespace {

__device__ __forceinline__ Smem &smem()
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    return *reinterpret_cast<Smem *>(smem_raw);
}

__global__ void __launch_bounds__(NT) k_fill_u64(u64 *p, u64 n, u64 v)
{
    for (u64 i = (u64)blockIdx.x * NT + threadIdx.x; i < n; i += (u64)gridDim.x * NT) p[i] = v;
}

// One heap operation followed by the resolution schedule (heapop.cuh).
__global__ void __launch_bounds__(NT) k_pbh_op(Scratch sc, HeapState *g_hs, HeapCounters *cnt, int op,
                                                const u32 *keys, const u32 *prios, u32 count, u32 r, u32 *kout,
                                                u32 *pout, u32 *nout)
{
    Smem &S = smem();
    GridTeam t{sc};
    t.init();
    if (threadIdx.x == 0) g_err_sink_set(sc.err, sc.bar);
    heap_op(t, S, g_hs, cnt, op, keys, prios, count, r, kout, pout, nout);
}

// Debug check of the heap invariants (one CTA; heapop.cuh).
__global__ void __launch_bounds__(NT) k_pbh_validate(const HeapState *g_hs, u32 *viol, u64 *stored, u64 *nvalid,
                                                      u32 *seen, u32 *dup)
{
    Smem &S = smem();
    if (threadIdx.x == 0) g_err_sink_set(nullptr);
    heap_validate(S, g_hs, viol, stored, nvalid, seen, dup);
}

} // namespace

namespace pbhk {
const void *kfn_fill_u64() { return reinterpret_cast<const void *>(&k_fill_u64); }
const void *kfn_pbh_op() { return reinterpret_cast<const void *>(&k_pbh_op); }
const void *kfn_pbh_validate() { return reinterpret_cast<const void *>(&k_pbh_validate); }
} // namespace pbhk
