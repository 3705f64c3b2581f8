// pbh.cu -- the C ABI (include/pbh.h) of the GB300 parallel bucket heap and
// parDijkstra: argument checks, workspace planning, launches.  The kernels
// are in k_*.cu (one translation unit each), their device code in core.cuh.
//
// Launch structure
//   pbh_*       one cooperative launch per heap operation (GridTeam over the
//               whole GPU): the operation, then Resolve(0) and the Theorem 3
//               schedule, all inside the launch.
//   sssp_run    one cooperative launch for the whole query (every round of
//               Section 4.1 runs inside it), or one CTA when opts->cta == 1.
//   sssp_batch  one persistent launch; each CTA pulls queries off a device
//               work queue and runs each with its own heap (CtaTeam).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pbh.h"
#include "kernels.h"
#include "plan.h"

using namespace pbhk;

// ================================================================= host

namespace {

thread_local std::string g_last_error = "";

pbh_status fail(pbh_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

pbh_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(PBH_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(x)                                              \
    do {                                                         \
        cudaError_t e_ = (x);                                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, #x);         \
    } while (0)


struct DevInfo {
    int sms = 0;
    int grid_op = 0, grid_ops = 0, grid_sssp = 0, max_sssp_per_sm = 1;
    bool ok = false;
};

DevInfo &devinfo()
{
    static std::mutex mu;
    static DevInfo info[64];
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    DevInfo &d = info[dev & 63];
    if (!d.ok) {
        cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        const size_t sm = sizeof(Smem);
        for (const void *k : {kfn_pbh_op(), kfn_sssp_grid(), kfn_sssp_cta(), kfn_sssp_batch(), kfn_pbh_validate(),
                              kfn_sssp_cluster(), kfn_serve(), kfn_sssp_batch_cluster(), kfn_pbh_ops(),
                              kfn_serve_cluster()})
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        for (const void *k : {kfn_sssp_cluster(), kfn_sssp_batch_cluster(), kfn_serve_cluster()})
            cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        int b1 = 0, b2 = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, kfn_pbh_op(), NT, sm);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, kfn_sssp_grid(), NT, sm);
        const int cap = 2; // CTAs per SM in a grid team: more only lengthen barriers
        d.grid_op = d.sms * std::max(1, std::min(b1, cap));
        int b3 = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b3, kfn_pbh_ops(), NT, sm);
        d.grid_ops = d.sms * std::max(1, std::min(b3, cap));
        if (d.grid_ops > (int)MAXGRID) d.grid_ops = (int)MAXGRID;
        d.grid_sssp = d.sms * 1; // one CTA per SM measured fastest (fewer barrier arrivals)
        d.max_sssp_per_sm = std::max(1, b2);
        if (d.grid_op > (int)MAXGRID) d.grid_op = (int)MAXGRID;
        if (d.grid_sssp > (int)MAXGRID) d.grid_sssp = (int)MAXGRID;
        d.ok = true;
    }
    return d;
}

constexpr u32 DEFAULT_R = 512;
constexpr u32 DEFAULT_D = 65536;

// Graphs of at most this many arcs run on one cluster when the caller
// leaves the team to the library (measured on GB300: a 64x64 and a 256x256
// grid are fastest on a 16-CTA cluster, banded graphs of 2^20 arcs and more
// on the whole GPU).
constexpr u64 AUTO_CLUSTER_MAX_ARCS = 1ull << 19;
constexpr u32 AUTO_CLUSTER = 16;

void resolve_opts(const sssp_opts *o, u32 *r, u32 *d, u32 *cta, u64 m = ~0ull)
{
    *r = (o && o->r) ? o->r : DEFAULT_R;
    *d = (o && o->d) ? o->d : DEFAULT_D;
    *cta = o ? o->cta : (m <= AUTO_CLUSTER_MAX_ARCS ? AUTO_CLUSTER : 0);
}

} // namespace

struct pbh {
    Plan plan;
    char *ws = nullptr;
    cudaStream_t stream = nullptr;
    int grid = 0;
    u32 d = 0;
    u32 key_space = 0;
};

extern "C" {

const char *pbh_last_error(void) { return g_last_error.c_str(); }

const char *pbh_version(void) { return "pbh-gb300 0.1 (sm_103a)"; }

size_t pbh_workspace_bytes(const pbh_params *p)
{
    if (!p || p->d == 0 || p->key_space == 0 || p->key_space > (1u << 31)) return 0;
    Plan plan;
    const u64 cap = p->capacity ? p->capacity : p->key_space;
    if (!plan_heap(nullptr, p->key_space, p->d, cap, nullptr, MAXGRID, &plan, true)) return 0;
    return plan.bytes;
}

pbh_status pbh_create(pbh_t **out, const pbh_params *p, void *ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!out || !p || !ws) return fail(PBH_E_INVAL, "pbh_create: null argument");
    if (p->d == 0 || p->key_space == 0 || p->key_space > (1u << 31))
        return fail(PBH_E_INVAL, "pbh_create: need d >= 1 and 1 <= key_space <= 2^31");
    if (reinterpret_cast<uintptr_t>(ws) % ALIGN) return fail(PBH_E_INVAL, "pbh_create: workspace not 256-byte aligned");
    const size_t need = pbh_workspace_bytes(p);
    if (need == 0) return fail(PBH_E_INVAL, "pbh_create: parameters give too many levels");
    if (ws_bytes < need) return fail(PBH_E_NOMEM, "pbh_create: workspace too small");
    DevInfo &di = devinfo();
    pbh *h = new pbh();
    const u64 cap = p->capacity ? p->capacity : p->key_space;
    plan_heap(static_cast<char *>(ws), p->key_space, p->d, cap, nullptr, MAXGRID, &h->plan, true);
    h->plan.hs.reset_on_extract = 1;
    h->plan.hs.keymask = 0xffffffffull;
    h->ws = static_cast<char *>(ws);
    h->stream = stream;
    h->grid = di.grid_op;
    h->d = p->d;
    h->key_space = p->key_space;
    cudaError_t e = cudaMemsetAsync(ws, 0, HDR_BYTES, stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->ws + OFF_HS, &h->plan.hs, sizeof(HeapState), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) {
        u64 *ptr = h->plan.cur, cnt = p->key_space, val = INF;
        void *fa[] = {&ptr, &cnt, &val};
        e = cudaLaunchKernel(kfn_fill_u64(), dim3(std::max(1, di.sms * 4)), dim3(NT), fa, 0, stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream); // the host copy of the state is on the stack
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "pbh_create");
    }
    *out = h;
    return PBH_OK;
}

static pbh_status launch_op(pbh_t *h, int op, const uint32_t *keys, const uint32_t *prios, uint32_t count, uint32_t r,
                            uint32_t *kout, uint32_t *pout, uint32_t *nout)
{
    Scratch sc = h->plan.sc;
    HeapState *g_hs = reinterpret_cast<HeapState *>(h->ws + OFF_HS);
    HeapCounters *cnt = reinterpret_cast<HeapCounters *>(h->ws + OFF_CNT);
    void *args[] = {&sc, &g_hs, &cnt, &op, &keys, &prios, &count, &r, &kout, &pout, &nout};
    cudaError_t e = cudaLaunchCooperativeKernel(kfn_pbh_op(), dim3(h->grid), dim3(NT), args, sizeof(Smem),
                                                h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "pbh op launch");
    return PBH_OK;
}

static_assert(sizeof(pbh_op) == sizeof(OpDesc), "pbh_op and the device descriptor share one layout");

pbh_status pbh_run_ops(pbh_t *h, const pbh_op *ops, uint32_t nops, uint32_t deep_ctas)
{
    if (!h || (!ops && nops)) return fail(PBH_E_INVAL, "pbh_run_ops: null argument");
    for (u32 k = 0; k < nops; k++) {
        const pbh_op &o = ops[k];
        if (o.kind == PBH_OP_BULK_UPDATE) {
            if (o.count > h->d) return fail(PBH_E_INVAL, "pbh_run_ops: count > d in operation " + std::to_string(k));
            if (o.count && (!o.d_keys || !o.d_prios))
                return fail(PBH_E_INVAL, "pbh_run_ops: null input in operation " + std::to_string(k));
        } else if (o.kind == PBH_OP_EXTRACT) {
            if (o.r > h->d) return fail(PBH_E_INVAL, "pbh_run_ops: r > d in operation " + std::to_string(k));
            if (!o.d_count_out || (o.r && (!o.d_keys_out || !o.d_prios_out)))
                return fail(PBH_E_INVAL, "pbh_run_ops: null output in operation " + std::to_string(k));
        } else {
            return fail(PBH_E_INVAL, "pbh_run_ops: unknown kind in operation " + std::to_string(k));
        }
    }
    const u32 grid = (u32)devinfo().grid_ops;
    const u32 nB = std::min<u32>(deep_ctas, grid / 2);
    u32 nA = grid - nB;
    Scratch scA = h->plan.sc;
    scA.bar = reinterpret_cast<u64 *>(h->ws + OFF_BAR_A);
    Scratch scB = h->plan.sc2;
    HeapState *g_hs = reinterpret_cast<HeapState *>(h->ws + OFF_HS);
    HeapCounters *cnt = reinterpret_cast<HeapCounters *>(h->ws + OFF_CNT);
    DeepSync *ds = reinterpret_cast<DeepSync *>(h->ws + OFF_DEEP);
    for (u32 k0 = 0; k0 < nops; k0 += OPS_MAX) {
        u32 nk = std::min<u32>(OPS_MAX, nops - k0);
        const OpDesc *dops = h->plan.ops;
        // the group barriers (their sizes may differ from call to call) and
        // the hand-over words start from zero in every launch
        CUDA_TRY(cudaMemsetAsync(h->ws + OFF_BAR_A, 0, OFF_DEEP + sizeof(DeepSync) - OFF_BAR_A, h->stream));
        CUDA_TRY(cudaMemcpyAsync(const_cast<OpDesc *>(dops), ops + k0, sizeof(OpDesc) * nk, cudaMemcpyHostToDevice,
                                 h->stream));
        void *args[] = {&scA, &scB, &g_hs, &cnt, &dops, &nk, &nA, &ds};
        cudaError_t e = cudaLaunchCooperativeKernel(kfn_pbh_ops(), dim3(grid), dim3(NT), args, sizeof(Smem),
                                                    h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "pbh_run_ops launch");
    }
    return PBH_OK;
}

pbh_status pbh_bulk_update(pbh_t *h, const uint32_t *d_keys, const uint32_t *d_prios, uint32_t count)
{
    if (!h) return fail(PBH_E_INVAL, "pbh_bulk_update: null handle");
    if (count == 0) return PBH_OK;
    if (!d_keys || !d_prios) return fail(PBH_E_INVAL, "pbh_bulk_update: null array");
    if (count > h->d) return fail(PBH_E_INVAL, "pbh_bulk_update: count > d");
    return launch_op(h, OP_BULK, d_keys, d_prios, count, 0, nullptr, nullptr, nullptr);
}

pbh_status pbh_assign(pbh_t *h, const uint32_t *d_keys, const uint32_t *d_prios, uint32_t count)
{
    if (!h) return fail(PBH_E_INVAL, "pbh_assign: null handle");
    if (count == 0) return PBH_OK;
    if (!d_keys || !d_prios) return fail(PBH_E_INVAL, "pbh_assign: null array");
    if (count > h->d) return fail(PBH_E_INVAL, "pbh_assign: count > d");
    return launch_op(h, OP_ASSIGN, d_keys, d_prios, count, 0, nullptr, nullptr, nullptr);
}

pbh_status pbh_delete(pbh_t *h, const uint32_t *d_keys, uint32_t count)
{
    if (!h) return fail(PBH_E_INVAL, "pbh_delete: null handle");
    if (count == 0) return PBH_OK;
    if (!d_keys) return fail(PBH_E_INVAL, "pbh_delete: null array");
    if (count > h->d) return fail(PBH_E_INVAL, "pbh_delete: count > d");
    return launch_op(h, OP_DELETE, d_keys, nullptr, count, 0, nullptr, nullptr, nullptr);
}

pbh_status pbh_extract_min(pbh_t *h, uint32_t r, uint32_t *d_keys_out, uint32_t *d_prios_out, uint32_t *d_count_out)
{
    if (!h || !d_count_out) return fail(PBH_E_INVAL, "pbh_extract_min: null argument");
    if (r > h->d) return fail(PBH_E_INVAL, "pbh_extract_min: r > d");
    if (r == 0) {
        cudaError_t e = cudaMemsetAsync(d_count_out, 0, sizeof(uint32_t), h->stream);
        return e == cudaSuccess ? PBH_OK : cuda_fail(e, "pbh_extract_min");
    }
    if (!d_keys_out || !d_prios_out) return fail(PBH_E_INVAL, "pbh_extract_min: null output");
    return launch_op(h, OP_EXTRACT, nullptr, nullptr, 0, r, d_keys_out, d_prios_out, d_count_out);
}

static pbh_status latched(const char *ws, cudaStream_t s)
{
    u32 err[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(err, ws + OFF_ERR, sizeof(err), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (err[0])
        return fail((pbh_status)err[0], "device reported an error (latched status, site " + std::to_string(err[1]) + ")");
    return PBH_OK;
}

pbh_status pbh_sync(pbh_t *h)
{
    if (!h) return fail(PBH_E_INVAL, "pbh_sync: null handle");
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return latched(h->ws, h->stream);
}

pbh_status pbh_size(pbh_t *h, uint64_t *out)
{
    if (!h || !out) return fail(PBH_E_INVAL, "pbh_size: null argument");
    HeapCounters c;
    CUDA_TRY(cudaMemcpyAsync(&c, h->ws + OFF_CNT, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    pbh_status s = latched(h->ws, h->stream);
    *out = c.inserted - c.extracted - c.deleted;
    return s;
}

pbh_status pbh_validate(pbh_t *h, uint32_t *viol, uint64_t *stored)
{
    if (!h || !viol || !stored) return fail(PBH_E_INVAL, "pbh_validate: null argument");
    u64 *tmp = reinterpret_cast<u64 *>(h->ws + OFF_RES + 8 * 8); // res[8..11] are free between ops
    CUDA_TRY(cudaMemsetAsync(tmp, 0, 3 * 8, h->stream));
    const size_t words = (h->key_space + 31) / 32;
    CUDA_TRY(cudaMemsetAsync(h->plan.seen, 0, 2 * 4 * words, h->stream));
    {
        const HeapState *ghs = reinterpret_cast<const HeapState *>(h->ws + OFF_HS);
        u32 *viol_d = reinterpret_cast<u32 *>(tmp);
        u64 *st_d = tmp + 1, *nv_d = tmp + 2;
        u32 *seen = h->plan.seen, *dup = h->plan.seen + words;
        void *va[] = {&ghs, &viol_d, &st_d, &nv_d, &seen, &dup};
        CUDA_TRY(cudaLaunchKernel(kfn_pbh_validate(), dim3(1), dim3(NT), va, sizeof(Smem), h->stream));
    }
    u64 v[3];
    HeapCounters c;
    CUDA_TRY(cudaMemcpyAsync(v, tmp, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(&c, h->ws + OFF_CNT, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    u32 bad = (u32)v[0];
    if (v[2] != c.inserted - c.extracted - c.deleted) bad |= 16; // every live key stored (valid) at least once
    *viol = bad;
    *stored = v[1];
    return latched(h->ws, h->stream);
}

pbh_status pbh_destroy(pbh_t *h)
{
    if (!h) return PBH_OK;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    delete h;
    return e == cudaSuccess ? PBH_OK : cuda_fail(e, "pbh_destroy");
}

// ------------------------------------------------------------------ SSSP

size_t sssp_workspace_bytes(uint32_t n, const sssp_opts *opts)
{
    u32 r, d, cta;
    resolve_opts(opts, &r, &d, &cta);
    if (n == 0) return HDR_BYTES;
    Plan plan;
    if (!plan_heap(nullptr, n, d, n, reinterpret_cast<u64 *>(8), MAXGRID, &plan)) return 0;
    return plan.bytes;
}

static pbh_status sssp_launch(const csr_t *g, const uint32_t *w, uint32_t source, uint64_t *dist, const sssp_opts *opts,
                              void *ws, size_t ws_bytes, cudaStream_t stream)
{
    u32 r, d, cta;
    if (!g || !dist || !ws) return fail(PBH_E_INVAL, "sssp_run: null argument");
    resolve_opts(opts, &r, &d, &cta, g->m);
    if (reinterpret_cast<uintptr_t>(ws) % ALIGN) return fail(PBH_E_INVAL, "sssp_run: workspace not 256-byte aligned");
    if (g->n == 0) {
        CUDA_TRY(cudaMemsetAsync(ws, 0, HDR_BYTES, stream));
        return PBH_OK;
    }
    if (!g->row_ptr || (g->m && (!g->col || !w))) return fail(PBH_E_INVAL, "sssp_run: null graph array");
    if (source >= g->n) return fail(PBH_E_INVAL, "sssp_run: source >= n");
    if (cta > MAXGRID) return fail(PBH_E_INVAL, "sssp_run: cta must be 0 (whole GPU), 1 (one CTA), 2..16 (cluster) "
                                                "or a grid of at most 4096 CTAs");
    const size_t need = sssp_workspace_bytes(g->n, opts);
    if (need == 0) return fail(PBH_E_INVAL, "sssp_run: options give too many levels");
    if (ws_bytes < need) return fail(PBH_E_NOMEM, "sssp_run: workspace too small");
    DevInfo &di = devinfo();
    Plan plan;
    plan_heap(static_cast<char *>(ws), g->n, d, g->n, reinterpret_cast<u64 *>(dist), MAXGRID, &plan);
    const u32 kb = key_bits(g->n);
    plan.hs.reset_on_extract = 0;
    plan.hs.keymask = (1ull << kb) - 1;
    plan.hs.settle = opts && (opts->flags & SSSP_SETTLE) ? 1 : 0;
    Graph gg{g->n, g->m, reinterpret_cast<const u64 *>(g->row_ptr), g->col, w};
    CUDA_TRY(cudaMemsetAsync(ws, 0, HDR_BYTES, stream));
    Scratch sc = plan.sc;
    sc.wait_ns = opts ? 1000ull * opts->wait_us : 0;
    sc.stall = opts && (opts->flags & SSSP_DEBUG_STALL) ? 1u : 0u;
    HeapState hs = plan.hs;
    u64 limit_ns = opts ? 1000000ull * opts->limit_ms : 0;
    const size_t smem_big = sizeof(Smem);
    void *args[] = {&sc, &hs, &gg, &source, &dist, &r, const_cast<u32 *>(&kb), &limit_ns};
    cudaError_t e;
    if (cta == 1) {
        e = cudaLaunchKernel(kfn_sssp_cta(), dim3(1), dim3(NT), args, sizeof(Smem), stream);
    } else if (cta >= 2 && cta <= 16) {
        // one thread-block cluster of `cta` CTAs (hardware cluster barrier)
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cta);
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = smem_big;
        cfg.stream = stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cta;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelExC(&cfg, kfn_sssp_cluster(), args);
    } else {
        // a cooperative grid: cta >= 17 CTAs, or the whole GPU with flags
        // bits 0-3 CTAs per SM (0 = one per SM)
        int per_sm = opts ? (int)(opts->flags & 15u) : 0;
        int grid = per_sm ? di.sms * std::min(per_sm, di.max_sssp_per_sm) : di.grid_sssp;
        if (cta > 16) {
            if ((int)cta > di.sms * di.max_sssp_per_sm)
                return fail(PBH_E_INVAL, "sssp_run: more CTAs than can be resident at once");
            grid = (int)cta;
        }
        if (grid > (int)MAXGRID) grid = (int)MAXGRID;
        e = cudaLaunchCooperativeKernel(kfn_sssp_grid(), dim3(grid), dim3(NT), args, smem_big, stream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "sssp launch");
    return PBH_OK;
}

pbh_status sssp_run(const csr_t *g, const uint32_t *d_weights, uint32_t source, uint64_t *d_dist_out,
                    const sssp_opts *opts, void *d_workspace, size_t ws_bytes, cudaStream_t stream)
{
    return sssp_launch(g, d_weights, source, d_dist_out, opts, d_workspace, ws_bytes, stream);
}

// ------------------------------------------------- allocation-free variant
//
// Some callers cannot allocate device memory at the point where they need a
// shortest-path query: code running under a custom allocator or a memory
// budget that forbids new allocations, plugins that must not grow the
// process's device footprint after start-up, or paths where a cudaMalloc
// would synchronise the device at a bad moment.  sssp_run_noalloc serves
// them: it runs the same query kernel as sssp_run, but its workspace is the
// file-scope array below instead of caller memory, so it calls no cudaMalloc,
// cudaFree or allocating library routine.
//
// The array is allocated once per device when the library's module is
// loaded on that device and stays allocated until the process exits.  Every
// call shares it and it keeps the previous call's contents; sssp_launch
// clears the header (status, counters, barrier) and the kernel initialises
// every other word it reads, so nothing stale leaks into a result.  Calls
// that overlap on the GPU (different streams, or different host threads)
// race on the array.

constexpr size_t NOALLOC_SCRATCH_BYTES = 32ull << 20; // 32 MiB per device

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64] = {};
} // namespace

pbh_status sssp_run_noalloc(const csr_t *g, const uint32_t *d_weights, uint32_t source, uint64_t *d_dist_out,
                            const sssp_opts *opts, cudaStream_t stream)
{
    if (!g) return fail(PBH_E_INVAL, "sssp_run_noalloc: null graph");
    const size_t need = sssp_workspace_bytes(g->n, opts);
    if (need == 0) return fail(PBH_E_INVAL, "sssp_run_noalloc: options give too many levels");
    if (need > NOALLOC_SCRATCH_BYTES)
        return fail(PBH_E_NOMEM, "sssp_run_noalloc: the query needs " + std::to_string(need) +
                                     " bytes of workspace; the static scratch holds " +
                                     std::to_string(NOALLOC_SCRATCH_BYTES) + " (use sssp_run with caller memory)");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(PBH_E_INVAL, "sssp_run_noalloc: device ordinal out of range");
    void *ws = nullptr;
    {
        // set-up once per device, with that device current: in host code the
        // array's name is only a stand-in, the kernel needs its device address
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "sssp_run_noalloc: cudaGetSymbolAddress");
            g_noalloc_ptr[dev] = p;
        }
        ws = g_noalloc_ptr[dev];
    }
    pbh_status st = sssp_launch(g, d_weights, source, d_dist_out, opts, ws, NOALLOC_SCRATCH_BYTES, stream);
    if (st != PBH_OK) return st;
    // wait for the query and return its latched device status (a 4-byte copy
    // into a stack variable; nothing is allocated)
    return latched(static_cast<const char *>(ws), stream);
}

size_t sssp_host_workspace_bytes(uint32_t n, uint64_t m, const sssp_opts *opts)
{
    size_t b = align_up(sssp_workspace_bytes(n, opts));
    b += align_up(8ull * (n + 1)) + 2 * align_up(4ull * m + 4) + align_up(8ull * n + 8);
    return b;
}

pbh_status sssp_run_host(uint32_t n, uint64_t m, const uint64_t *h_row_ptr, const uint32_t *h_col,
                         const uint32_t *h_weights, uint32_t source, uint64_t *h_dist_out, const sssp_opts *opts,
                         void *d_workspace, size_t ws_bytes, cudaStream_t stream)
{
    if (!h_row_ptr || !h_dist_out || !d_workspace || (m && (!h_col || !h_weights)))
        return fail(PBH_E_INVAL, "sssp_run_host: null argument");
    if (ws_bytes < sssp_host_workspace_bytes(n, m, opts)) return fail(PBH_E_NOMEM, "sssp_run_host: workspace too small");
    char *p = static_cast<char *>(d_workspace);
    size_t off = align_up(sssp_workspace_bytes(n, opts));
    uint64_t *rp = reinterpret_cast<uint64_t *>(p + off);
    off += align_up(8ull * (n + 1));
    uint32_t *col = reinterpret_cast<uint32_t *>(p + off);
    off += align_up(4ull * m + 4);
    uint32_t *w = reinterpret_cast<uint32_t *>(p + off);
    off += align_up(4ull * m + 4);
    uint64_t *dist = reinterpret_cast<uint64_t *>(p + off);
    CUDA_TRY(cudaMemcpyAsync(rp, h_row_ptr, 8ull * (n + 1), cudaMemcpyHostToDevice, stream));
    if (m) {
        CUDA_TRY(cudaMemcpyAsync(col, h_col, 4ull * m, cudaMemcpyHostToDevice, stream));
        CUDA_TRY(cudaMemcpyAsync(w, h_weights, 4ull * m, cudaMemcpyHostToDevice, stream));
    }
    csr_t g{n, m, rp, col};
    pbh_status s = sssp_launch(&g, w, source, dist, opts, d_workspace, ws_bytes, stream);
    if (s != PBH_OK) return s;
    CUDA_TRY(cudaMemcpyAsync(h_dist_out, dist, 8ull * n, cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaStreamSynchronize(stream));
    return latched(p, stream);
}

pbh_status sssp_stats(const void *ws, sssp_stats_t *out, cudaStream_t stream)
{
    if (!ws || !out) return fail(PBH_E_INVAL, "sssp_stats: null argument");
    u64 st[STAT_N];
    u32 err2[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(st, ws, sizeof(st), cudaMemcpyDeviceToHost, stream));
    CUDA_TRY(cudaMemcpyAsync(err2, static_cast<const char *>(ws) + OFF_ERR, 8, cudaMemcpyDeviceToHost, stream));
    const u32 err = err2[0];
    CUDA_TRY(cudaStreamSynchronize(stream));
    memset(out, 0, sizeof(*out));
    out->rounds = st[STAT_ROUNDS];
    out->extracted = st[STAT_EXTRACTED];
    out->relaxations = st[STAT_RELAX];
    out->improvements = st[STAT_IMPROVE];
    out->stale_dropped = st[STAT_STALE];
    out->merged = st[STAT_MERGED];
    for (int i = 0; i < 16 && i < MAXQ; i++) out->resolves[i] = st[STAT_RES0 + i];
    out->t_relax_ns = st[STAT_T_RELAX];
    out->t_sort_ns = st[STAT_T_SORT];
    out->t_empty0_ns = st[STAT_T_EMPTY];
    out->t_fill0_ns = st[STAT_T_FILL];
    out->t_deeper_ns = st[STAT_T_DEEP];
    out->t_ensure_ns = st[STAT_T_ENSURE];
    out->barriers = st[STAT_SYNCS];
    out->levels = (u32)st[STAT_LEVELS];
    out->r_eff = (u32)st[STAT_REFF];
    out->max_degree = (u32)st[STAT_MAXDEG];
    out->status = err;
    out->settled = st[STAT_SETTLED];
    if (err)
        return fail((pbh_status)err, "sssp: device reported an error (latched status, site " +
                                         std::to_string(err2[1]) + ")");
    return PBH_OK;
}

pbh_status pbh_stats(pbh_t *h, sssp_stats_t *out)
{
    if (!h || !out) return fail(PBH_E_INVAL, "pbh_stats: null argument");
    return sssp_stats(h->ws, out, h->stream);
}

// --------------------------------------------------------------- batched

namespace {
// Batch workspace: one claim counter per team size (0 and 1: one CTA; 2..16:
// a cluster of that many CTAs), the query descriptors, the run order, then
// one heap region per query.
constexpr u32 BATCH_COUNTERS = 32;

struct BatchPlan {
    size_t bytes = 0;
    size_t off_desc = 0, off_order = 0, off_next = 0;
    std::vector<size_t> q_off;
};

u32 query_team(const sssp_query &q) { return q.cta >= 2 ? q.cta : 1; }

bool plan_batch(const sssp_query *qs, uint32_t nq, BatchPlan *bp)
{
    size_t off = align_up(sizeof(u32) * BATCH_COUNTERS);
    bp->off_next = 0;
    bp->off_desc = off;
    off = align_up(off + sizeof(QueryDesc) * nq);
    bp->off_order = off;
    off = align_up(off + sizeof(u32) * nq);
    bp->q_off.resize(nq);
    for (u32 i = 0; i < nq; i++) {
        const u32 d = qs[i].d ? qs[i].d : DEFAULT_D;
        if (qs[i].cta > 16) return false;
        Plan p;
        const u32 n = std::max<u32>(qs[i].g.n, 1);
        if (!plan_heap(nullptr, n, d, n, reinterpret_cast<u64 *>(8), query_team(qs[i]), &p)) return false;
        bp->q_off[i] = off;
        off = align_up(off + p.bytes + sizeof(HeapState));
    }
    bp->bytes = off;
    return true;
}

// A second stream per device for the cluster launch of a batch, forked from
// and joined back to the caller's stream with events.
cudaStream_t side_stream()
{
    static std::mutex mu;
    static cudaStream_t st[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!st[dev & 63]) cudaStreamCreateWithFlags(&st[dev & 63], cudaStreamNonBlocking);
    return st[dev & 63];
}
} // namespace

size_t sssp_batch_workspace_bytes(const sssp_query *qs, uint32_t nq)
{
    if (!qs && nq) return 0;
    BatchPlan bp;
    if (!plan_batch(qs, nq, &bp)) return 0;
    return bp.bytes;
}

pbh_status sssp_batch_run(const sssp_query *qs, uint32_t nq, void *ws, size_t ws_bytes, cudaStream_t stream)
{
    if (!ws || (!qs && nq)) return fail(PBH_E_INVAL, "sssp_batch_run: null argument");
    if (reinterpret_cast<uintptr_t>(ws) % ALIGN) return fail(PBH_E_INVAL, "sssp_batch_run: workspace not aligned");
    if (nq == 0) return PBH_OK;
    BatchPlan bp;
    if (!plan_batch(qs, nq, &bp)) return fail(PBH_E_INVAL, "sssp_batch_run: bad team (cta > 16) or too many levels");
    if (ws_bytes < bp.bytes) return fail(PBH_E_NOMEM, "sssp_batch_run: workspace too small");
    char *base = static_cast<char *>(ws);
    std::vector<QueryDesc> desc(nq);
    std::vector<HeapState> states(nq);
    std::vector<u64> work(nq);
    for (u32 i = 0; i < nq; i++) {
        const sssp_query &q = qs[i];
        if (q.g.n == 0 || !q.g.row_ptr || !q.d_dist_out || (q.g.m && (!q.g.col || !q.d_weights)) || q.source >= q.g.n)
            return fail(PBH_E_INVAL, "sssp_batch_run: bad query " + std::to_string(i));
        const u32 r = q.r ? q.r : DEFAULT_R, d = q.d ? q.d : DEFAULT_D;
        Plan p;
        char *qb = base + bp.q_off[i];
        plan_heap(qb, q.g.n, d, q.g.n, reinterpret_cast<u64 *>(q.d_dist_out), query_team(q), &p);
        const u32 kb = key_bits(q.g.n);
        p.hs.reset_on_extract = 0;
        p.hs.keymask = (1ull << kb) - 1;
        states[i] = p.hs;
        QueryDesc &qd = desc[i];
        qd.sc = p.sc;
        qd.hs = reinterpret_cast<HeapState *>(qb + p.bytes);
        qd.g = Graph{q.g.n, q.g.m, reinterpret_cast<const u64 *>(q.g.row_ptr), q.g.col, q.d_weights};
        qd.dist = reinterpret_cast<u64 *>(q.d_dist_out);
        qd.source = q.source;
        qd.r = r;
        qd.kb = kb;
        qd.header = reinterpret_cast<u64 *>(qb);
        qd.header_words = 1024 / 8; // stats, status, counters, results (not the state copy)
        work[i] = (u64)q.g.n + q.g.m;
    }
    // the run order: queries grouped by team size, largest first within a
    // group (longest-processing-time order); group k starts at first[k]
    std::vector<u32> order(nq);
    for (u32 i = 0; i < nq; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](u32 a, u32 b) {
        const u32 ta = query_team(qs[a]), tb = query_team(qs[b]);
        return ta != tb ? ta < tb : work[a] > work[b];
    });
    u32 first[18] = {}, count[18] = {};
    u64 team_work[18] = {}, all_work = 0;
    for (u32 i = 0; i < nq; i++) {
        const u32 k = query_team(qs[order[i]]);
        if (count[k]++ == 0) first[k] = i;
        team_work[k] += work[order[i]];
        all_work += work[order[i]];
    }
    CUDA_TRY(cudaMemsetAsync(base + bp.off_next, 0, sizeof(u32) * BATCH_COUNTERS, stream));
    CUDA_TRY(cudaMemcpyAsync(base + bp.off_desc, desc.data(), sizeof(QueryDesc) * nq, cudaMemcpyHostToDevice, stream));
    CUDA_TRY(cudaMemcpyAsync(base + bp.off_order, order.data(), sizeof(u32) * nq, cudaMemcpyHostToDevice, stream));
    for (u32 i = 0; i < nq; i++)
        CUDA_TRY(cudaMemcpyAsync(desc[i].hs, &states[i], sizeof(HeapState), cudaMemcpyHostToDevice, stream));
    DevInfo &di = devinfo();
    const QueryDesc *qd = reinterpret_cast<const QueryDesc *>(base + bp.off_desc);
    const u32 *ord = reinterpret_cast<const u32 *>(base + bp.off_order);
    u32 *next = reinterpret_cast<u32 *>(base + bp.off_next);
    // cluster teams: one launch per cluster size on the side stream, each
    // with a share of the SMs in proportion to its share of the work (the
    // one-CTA launch on the caller's stream takes the rest as they free up)
    bool forked = false;
    cudaStream_t side = nullptr;
    for (u32 k = 2; k <= 16; k++) {
        if (!count[k]) continue;
        if (!forked) {
            side = side_stream();
            if (!side) return fail(PBH_E_CUDA, "sssp_batch_run: no side stream");
            cudaEvent_t fork;
            CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
            CUDA_TRY(cudaEventRecord(fork, stream));
            CUDA_TRY(cudaStreamWaitEvent(side, fork, 0));
            CUDA_TRY(cudaEventDestroy(fork));
            forked = true;
        }
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = k;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = sizeof(Smem);
        cfg.stream = side;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cfg.gridDim = dim3(k);
        int fit = 0;
        CUDA_TRY(cudaOccupancyMaxActiveClusters(&fit, kfn_sssp_batch_cluster(), &cfg));
        const double share = all_work ? (double)team_work[k] / (double)all_work : 1.0;
        u32 clusters = (u32)std::max(1.0, share * di.sms / k + 0.5);
        clusters = std::min(clusters, count[k]);
        if (fit > 0) clusters = std::min(clusters, (u32)fit);
        cfg.gridDim = dim3(clusters * k);
        const u32 *ord_k = ord + first[k];
        u32 nq_k = count[k];
        u32 *next_k = next + k;
        void *ca[] = {&qd, &ord_k, &nq_k, &next_k};
        CUDA_TRY(cudaLaunchKernelExC(&cfg, kfn_sssp_batch_cluster(), ca));
    }
    if (count[1]) {
        int bps = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kfn_sssp_batch(), NT, sizeof(Smem));
        u32 grid = (u32)std::max(1, di.sms * std::max(1, bps));
        grid = std::min(grid, count[1]);
        const u32 *ord_1 = ord + first[1];
        u32 nq_1 = count[1];
        u32 *next_1 = next + 1;
        void *ba[] = {&qd, &ord_1, &nq_1, &next_1};
        CUDA_TRY(cudaLaunchKernel(kfn_sssp_batch(), dim3(grid), dim3(NT), ba, sizeof(Smem), stream));
    }
    if (forked) {
        cudaEvent_t join;
        CUDA_TRY(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
        CUDA_TRY(cudaEventRecord(join, side));
        CUDA_TRY(cudaStreamWaitEvent(stream, join, 0));
        CUDA_TRY(cudaEventDestroy(join));
    }
    // pageable source buffers: make sure the copies have consumed them
    CUDA_TRY(cudaStreamSynchronize(stream));
    return PBH_OK;
}

// ---------------------------------------------------------------- serving

struct pbh_server {
    ServeRecord *ring = nullptr; // pinned, mapped
    ServeCtl *ctl = nullptr;     // pinned, mapped
    u64 *done = nullptr, *t_begin = nullptr, *t_end = nullptr; // pinned, mapped
    u32 slots = 0;
    u64 next = 0;                // next ticket
    u64 *head = nullptr;         // device claim counter
    cudaStream_t stream = nullptr;
    bool running = false;
    u32 team = 1;                // CTAs per request: 1, or a cluster of 2..16
};

size_t srv_workspace_bytes(void) { return ALIGN; }

size_t srv_query_workspace_bytes(const sssp_query *q)
{
    if (!q || q->g.n == 0 || q->cta > 16) return 0;
    const u32 d = q->d ? q->d : DEFAULT_D;
    Plan p;
    if (!plan_heap(nullptr, q->g.n, d, q->g.n, reinterpret_cast<u64 *>(8), query_team(*q), &p)) return 0;
    return p.bytes;
}

pbh_status srv_create(pbh_server_t **out, uint32_t slots, uint32_t ctas, void *d_workspace, size_t ws_bytes,
                      cudaStream_t stream)
{
    return srv_create_team(out, slots, ctas, 1, d_workspace, ws_bytes, stream);
}

pbh_status srv_create_team(pbh_server_t **out, uint32_t slots, uint32_t ctas, uint32_t team, void *d_workspace,
                           size_t ws_bytes, cudaStream_t stream)
{
    if (!out || !d_workspace || slots == 0) return fail(PBH_E_INVAL, "srv_create: null argument or zero slots");
    if (ws_bytes < srv_workspace_bytes()) return fail(PBH_E_NOMEM, "srv_create: workspace too small");
    if (team == 0 || team > 16) return fail(PBH_E_INVAL, "srv_create_team: team must be 1..16");
    if (team > 1 && (ctas == 0 || ctas % team))
        return fail(PBH_E_INVAL, "srv_create_team: a cluster server needs ctas, a multiple of the team");
    DevInfo &di = devinfo();
    if (team > 1) {
        // every cluster must be resident at once (they wait for requests)
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = team;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(team);
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = sizeof(Smem);
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int fit = 0;
        CUDA_TRY(cudaOccupancyMaxActiveClusters(&fit, kfn_serve_cluster(), &cfg));
        if ((u32)fit < ctas / team)
            return fail(PBH_E_INVAL, "srv_create_team: only " + std::to_string(fit) + " clusters of " +
                                         std::to_string(team) + " can be resident");
    }
    pbh_server *sv = new pbh_server();
    sv->team = team;
    sv->slots = slots;
    sv->stream = stream;
    sv->head = static_cast<u64 *>(d_workspace);
    auto host_alloc = [&](void **p, size_t bytes) {
        cudaError_t e = cudaHostAlloc(p, bytes, cudaHostAllocMapped | cudaHostAllocPortable);
        if (e == cudaSuccess) memset(*p, 0, bytes);
        return e;
    };
    cudaError_t e = host_alloc(reinterpret_cast<void **>(&sv->ring), sizeof(ServeRecord) * slots);
    if (e == cudaSuccess) e = host_alloc(reinterpret_cast<void **>(&sv->ctl), sizeof(ServeCtl));
    if (e == cudaSuccess) e = host_alloc(reinterpret_cast<void **>(&sv->done), 8ull * slots);
    if (e == cudaSuccess) e = host_alloc(reinterpret_cast<void **>(&sv->t_begin), 8ull * slots);
    if (e == cudaSuccess) e = host_alloc(reinterpret_cast<void **>(&sv->t_end), 8ull * slots);
    if (e == cudaSuccess) e = cudaMemsetAsync(sv->head, 0, 8, stream);
    int bps = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kfn_serve(), NT, sizeof(Smem));
    if (e == cudaSuccess) {
        const u32 grid = ctas ? ctas : (u32)(di.sms * std::max(1, bps));
        // device-visible addresses of the mapped buffers (identical under unified addressing)
        ServeRecord *dring;
        ServeCtl *dctl;
        u64 *ddone, *dtb, *dte;
        e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&dring), sv->ring, 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&dctl), sv->ctl, 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&ddone), sv->done, 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&dtb), sv->t_begin, 0);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&dte), sv->t_end, 0);
        if (e == cudaSuccess) {
            u64 *head = sv->head;
            void *sa[] = {&dring, &dctl, &ddone, &dtb, &dte, &slots, &head};
            if (team == 1) {
                e = cudaLaunchKernel(kfn_serve(), dim3(grid), dim3(NT), sa, sizeof(Smem), stream);
            } else {
                cudaLaunchConfig_t cfg = {};
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeClusterDimension;
                attr[0].val.clusterDim.x = team;
                attr[0].val.clusterDim.y = 1;
                attr[0].val.clusterDim.z = 1;
                cfg.gridDim = dim3(ctas);
                cfg.blockDim = dim3(NT);
                cfg.dynamicSmemBytes = sizeof(Smem);
                cfg.stream = stream;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                e = cudaLaunchKernelExC(&cfg, kfn_serve_cluster(), sa);
            }
        }
    }
    if (e != cudaSuccess) {
        cudaFreeHost(sv->ring);
        cudaFreeHost(sv->ctl);
        cudaFreeHost(sv->done);
        cudaFreeHost(sv->t_begin);
        cudaFreeHost(sv->t_end);
        delete sv;
        return cuda_fail(e, "srv_create");
    }
    sv->running = true;
    *out = sv;
    return PBH_OK;
}

pbh_status srv_submit(pbh_server_t *sv, const sssp_query *q, void *d_query_ws, size_t ws_bytes, uint64_t *ticket)
{
    if (!sv || !q || !d_query_ws || !ticket) return fail(PBH_E_INVAL, "srv_submit: null argument");
    if (!sv->running) return fail(PBH_E_INVAL, "srv_submit: server stopped");
    if (q->g.n == 0 || !q->g.row_ptr || !q->d_dist_out || (q->g.m && (!q->g.col || !q->d_weights)) ||
        q->source >= q->g.n)
        return fail(PBH_E_INVAL, "srv_submit: bad query");
    if (reinterpret_cast<uintptr_t>(d_query_ws) % ALIGN) return fail(PBH_E_INVAL, "srv_submit: workspace not aligned");
    if (query_team(*q) != sv->team)
        return fail(PBH_E_INVAL, "srv_submit: the query's team (cta) differs from the server's");
    const size_t need = srv_query_workspace_bytes(q);
    if (need == 0 || ws_bytes < need) return fail(PBH_E_NOMEM, "srv_submit: query workspace too small");
    const u64 k = sv->next;
    const u32 slot = (u32)(k % sv->slots);
    if (k >= sv->slots && *(volatile u64 *)&sv->done[slot] != k - sv->slots + 1)
        return fail(PBH_E_CAPACITY, "srv_submit: ring slot still in use");
    const u32 d = q->d ? q->d : DEFAULT_D, r = q->r ? q->r : DEFAULT_R;
    Plan p;
    char *qb = static_cast<char *>(d_query_ws);
    plan_heap(qb, q->g.n, d, q->g.n, reinterpret_cast<u64 *>(q->d_dist_out), sv->team, &p);
    const u32 kb = key_bits(q->g.n);
    p.hs.reset_on_extract = 0;
    p.hs.keymask = (1ull << kb) - 1;
    ServeRecord &rec = sv->ring[slot];
    rec.hs = p.hs;
    QueryDesc qd{};
    qd.sc = p.sc;
    void *dhs = nullptr;
    if (cudaHostGetDevicePointer(&dhs, &rec.hs, 0) != cudaSuccess) return fail(PBH_E_CUDA, "srv_submit: mapping");
    qd.hs = static_cast<HeapState *>(dhs);
    qd.g = Graph{q->g.n, q->g.m, reinterpret_cast<const u64 *>(q->g.row_ptr), q->g.col, q->d_weights};
    qd.dist = reinterpret_cast<u64 *>(q->d_dist_out);
    qd.source = q->source;
    qd.r = r;
    qd.kb = kb;
    qd.header = reinterpret_cast<u64 *>(qb);
    qd.header_words = 1024 / 8;
    rec.q = qd;
    std::atomic_thread_fence(std::memory_order_seq_cst); // the record before the tail
    sv->next = k + 1;
    *(volatile u64 *)&sv->ctl->tail = k + 1;
    *ticket = k;
    return PBH_OK;
}

pbh_status srv_completion_arrays(pbh_server_t *sv, uint64_t **done, uint64_t **t_begin, uint64_t **t_end,
                                 uint32_t *slots)
{
    if (!sv || !done || !t_begin || !t_end || !slots) return fail(PBH_E_INVAL, "srv_completion_arrays: null argument");
    *done = reinterpret_cast<uint64_t *>(sv->done);
    *t_begin = reinterpret_cast<uint64_t *>(sv->t_begin);
    *t_end = reinterpret_cast<uint64_t *>(sv->t_end);
    *slots = sv->slots;
    return PBH_OK;
}

pbh_status srv_request_stop(pbh_server_t *sv)
{
    if (!sv) return fail(PBH_E_INVAL, "srv_request_stop: null server");
    *(volatile u32 *)&sv->ctl->stop = 1;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    return PBH_OK;
}

pbh_status srv_heartbeat(pbh_server_t *sv)
{
    if (!sv) return fail(PBH_E_INVAL, "srv_heartbeat: null server");
    *(volatile u64 *)&sv->ctl->heartbeat = *(volatile u64 *)&sv->ctl->heartbeat + 1;
    return PBH_OK;
}

pbh_status srv_idle_limit(pbh_server_t *sv, uint64_t ns)
{
    if (!sv) return fail(PBH_E_INVAL, "srv_idle_limit: null server");
    *(volatile u64 *)&sv->ctl->idle_ns = ns;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    return PBH_OK;
}

pbh_status srv_stop(pbh_server_t *sv)
{
    if (!sv) return fail(PBH_E_INVAL, "srv_stop: null server");
    if (sv->running) {
        *(volatile u32 *)&sv->ctl->stop = 1;
        std::atomic_thread_fence(std::memory_order_seq_cst);
        cudaError_t e = cudaStreamSynchronize(sv->stream);
        sv->running = false;
        if (e != cudaSuccess) return cuda_fail(e, "srv_stop");
    }
    const u32 st = *(volatile u32 *)&sv->ctl->status;
    if (st) return fail((pbh_status)st, "server: a CTA waited past the idle limit for a request");
    return PBH_OK;
}

pbh_status srv_destroy(pbh_server_t *sv)
{
    if (!sv) return PBH_OK;
    pbh_status s = srv_stop(sv);
    cudaFreeHost(sv->ring);
    cudaFreeHost(sv->ctl);
    cudaFreeHost(sv->done);
    cudaFreeHost(sv->t_begin);
    cudaFreeHost(sv->t_end);
    delete sv;
    return s;
}

pbh_status sssp_batch_status(const void *ws, uint32_t nq, uint32_t *h_status, uint64_t *h_rounds, cudaStream_t stream)
{
    if (!ws || (nq && !h_status)) return fail(PBH_E_INVAL, "sssp_batch_status: null argument");
    CUDA_TRY(cudaStreamSynchronize(stream));
    const char *base = static_cast<const char *>(ws);
    std::vector<QueryDesc> desc(nq);
    const size_t off_desc = align_up(sizeof(u32) * BATCH_COUNTERS);
    CUDA_TRY(cudaMemcpy(desc.data(), base + off_desc, sizeof(QueryDesc) * nq, cudaMemcpyDeviceToHost));
    pbh_status worst = PBH_OK;
    for (u32 i = 0; i < nq; i++) {
        u32 err[2] = {0, 0};
        u64 rounds = 0;
        const char *qb = reinterpret_cast<const char *>(desc[i].header);
        CUDA_TRY(cudaMemcpy(err, qb + OFF_ERR, 8, cudaMemcpyDeviceToHost));
        CUDA_TRY(cudaMemcpy(&rounds, qb + OFF_STATS + 8 * STAT_ROUNDS, 8, cudaMemcpyDeviceToHost));
        h_status[i] = err[0] | (err[1] << 16);
        if (h_rounds) h_rounds[i] = rounds;
        if (err[0] && worst == PBH_OK) worst = (pbh_status)err[0];
    }
    if (worst != PBH_OK) return fail(worst, "sssp_batch: a query reported an error");
    return PBH_OK;
}

} // extern "C"
