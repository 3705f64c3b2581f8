// kernels.h -- what the host ABI (pbh.cu) and the kernel translation units
// share: the records the kernels read, and one accessor per kernel that
// returns its entry point for the runtime's C launch API (cudaLaunchKernel,
// cudaLaunchCooperativeKernel, cudaLaunchKernelExC, cudaFuncSetAttribute).
//
// Every kernel lives in its own translation unit (k_*.cu) so that the
// library's kernels compile in parallel; their device code is core.cuh.
#pragma once
#include <cuda_runtime.h>

#include "core.cuh"

namespace pbhk {

// One query of the batched and served kernels.
struct QueryDesc {
    Scratch sc;
    HeapState *hs; // initial (empty) heap layout of the query
    Graph g;
    u64 *dist;
    u32 source, r, kb, pad;
    u64 *header;   // stats + status region to clear
    u64 header_words;
    u64 limit_ns;  // bound on the query's run time (0 = the default)
};

// Serving: a ring of request records in pinned, device-mapped host memory.
struct ServeRecord {
    QueryDesc q; // q.hs points at hs below (device-visible address of this slot)
    HeapState hs;
};

struct ServeCtl {
    u64 tail;   // requests published by the host (monotone)
    u32 stop;   // host: no more requests, wind down
    u32 status; // server: latched status (idle timeout)
    u64 claimed;
    u64 idle_ns;   // bound on how long the host may stay silent (0 = the default)
    u64 heartbeat; // host: advanced while the host is alive (srv_heartbeat)
    u64 pad[3];
};

// Default bound on a CTA's wait for a request: 60 s without any sign of the
// host (a new request or a heartbeat).
constexpr u64 SERVE_IDLE_NS = 60000000000ull;

// Entry points (host stubs) of the kernels, one translation unit each.
const void *kfn_fill_u64();     // (u64 *p, u64 n, u64 v)
const void *kfn_pbh_op();       // one heap operation + its resolves (cooperative grid)
const void *kfn_pbh_validate(); // debug check of the level invariants (one CTA)
const void *kfn_pbh_ops();      // a sequence of heap operations, concurrent level resolution
const void *kfn_sssp_grid();    // one query on the whole GPU (cooperative grid)
const void *kfn_sssp_cluster(); // one query on one thread-block cluster
const void *kfn_sssp_cta();     // one query on one CTA
const void *kfn_sssp_batch();   // many queries, one per CTA, one launch
const void *kfn_sssp_batch_cluster(); // many queries, one per thread-block cluster
const void *kfn_serve();        // the persistent server
const void *kfn_serve_cluster(); // the persistent server, one thread-block cluster per request

} // namespace pbhk
