// k_ops.cu -- a sequence of heap operations in one cooperative launch, with
// concurrent resolution of non-adjacent levels (concurrent.cuh).
//
// Device code: core.cuh, concurrent.cuh.  Host ABI: pbh.cu.
#include "kernels.h"
#include "concurrent.cuh"

using namespace pbhk;

namespace {

__device__ __forceinline__ Smem &smem()
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    return *reinterpret_cast<Smem *>(smem_raw);
}

// A sequence of heap operations in one cooperative launch with concurrent
// resolution of non-adjacent levels: CTAs [0, nA) form the operation group,
// the rest the deep group (concurrent.cuh).  With no deep group, or fewer
// than three levels, the operation group runs the whole schedule itself.
__global__ void __launch_bounds__(NT, 2) k_pbh_ops(Scratch scA, Scratch scB, HeapState *g_hs, HeapCounters *cnt,
                                                 const OpDesc *ops, u32 nops, u32 nA, DeepSync *ds)
{
    Smem &S = smem();
    const bool op_group = blockIdx.x < nA;
    GroupTeam t{op_group ? scA : scB, op_group ? 0u : nA, op_group ? nA : gridDim.x - nA};
    t.init();
    if (threadIdx.x == 0) g_err_sink_set(t.sc.err, t.sc.bar);
    state_load(S, g_hs);
    const bool deep = S.hs.q > 2 && nA < gridDim.x;
    if (op_group) {
        OpsCtl c{g_hs, ds, 0, deep, true, true, false};
        if (read_err(scA.err) != 0) { // a latched error makes the heap read-only
            if (blockIdx.x == 0 && threadIdx.x == 0) *(volatile u32 *)&ds->stop = 1;
            return;
        }
        run_ops(t, S, cnt, ops, nops, c);
    } else if (deep) {
        deep_serve(t, S, g_hs, ds);
    }
}

} // namespace

namespace pbhk {
const void *kfn_pbh_ops() { return reinterpret_cast<const void *>(&k_pbh_ops); }
} // namespace pbhk
