// Many parDijkstra queries in one emulated persistent launch, the body of
// k_sssp_batch: P emulated CTAs claim queries from a work queue (an atomic
// counter over the longest-first run order) and run each on its own heap
// with the one-CTA team (CtaTeam); or, with a cluster size C >= 2, the body
// of k_sssp_batch_cluster: P / C clusters, whose first CTA claims a query
// and the others read its number through distributed shared memory, each
// query on one cluster (ClusterTeam).  For the CPU tests.  Usage:
//   batch_harness QUERIES OUT P [C]
// QUERIES: u64 nq; per query u64 n, m, source, r, d; u64 row_ptr[n+1];
// u32 col[m]; u32 w[m].
// OUT: per query u64 status, u64 rounds, u64 levels, then u64 dist[n].
// Exits 0 (ok), 5 (a query latched a device error) or 7 (no thread made
// progress for 30 s: the emulated kernel is stuck).
#include "cuda_shim.h"
#include "core_host.h"
#include "kernels_host.h"
#include "plan_host.h"
#include <algorithm>
#include <vector>
using namespace pbhk;

struct Query {
    u32 n, source, r, d;
    u64 m;
    std::vector<u64> row_ptr, dist;
    std::vector<u32> col, w;
    Plan p;
    char *header = nullptr;
    HeapState *hs = nullptr; // the initial (empty) heap layout the query loads
};

int main(int argc, char **argv)
{
    if (argc < 4) return 1;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    uint64_t nq = 0;
    if (fread(&nq, 8, 1, f) != 1 || nq == 0 || nq > 4096) return 2;
    std::vector<Query> qs(nq);
    for (auto &q : qs) {
        uint64_t h[5];
        if (fread(h, 8, 5, f) != 5) return 3;
        q.n = (u32)h[0];
        q.m = h[1];
        q.source = (u32)h[2];
        q.r = (u32)h[3];
        q.d = (u32)h[4];
        if (q.n == 0 || q.source >= q.n || q.r == 0 || q.d == 0) return 3;
        q.row_ptr.resize(q.n + 1);
        q.col.resize(q.m + 1);
        q.w.resize(q.m + 1);
        q.dist.assign(q.n, 0xABABABABABABABABull);
        if (fread(q.row_ptr.data(), 8, q.n + 1, f) != q.n + 1 || fread(q.col.data(), 4, q.m, f) != q.m ||
            fread(q.w.data(), 4, q.m, f) != q.m)
            return 3;
    }
    fclose(f);
    const int P = atoi(argv[3]);
    const int C = argc > 4 ? atoi(argv[4]) : 1;
    if (P < 1 || P > 16 || C < 1 || P % C) return 1;
    gridDim.x = P;
    std::vector<void *> bufs;
    auto take = [&](size_t bytes) {
        void *p = malloc(bytes ? bytes : 8);
        memset(p, 0xAB, bytes);
        bufs.push_back(p);
        return (char *)p;
    };
    // the host side of sssp_batch_run: a heap per query over its distance
    // array, one-CTA teams, and the run order (largest n + m first)
    std::vector<QueryDesc> desc(nq);
    std::vector<u32> order(nq);
    for (u64 i = 0; i < nq; i++) {
        Query &q = qs[i];
        q.header = (char *)calloc(HDR_BYTES, 1);
        if (!plan_heap_with(take, q.header, q.n, q.d, q.n, q.dist.data(), C, &q.p)) return 4;
        const u32 kb = key_bits(q.n);
        q.p.hs.reset_on_extract = 0;
        q.p.hs.keymask = (1ull << kb) - 1;
        q.hs = (HeapState *)take(sizeof(HeapState));
        memcpy(q.hs, &q.p.hs, sizeof(HeapState));
        QueryDesc &qd = desc[i];
        qd.sc = q.p.sc;
        qd.hs = q.hs;
        qd.g = Graph{q.n, q.m, q.row_ptr.data(), q.col.data(), q.w.data()};
        qd.dist = q.dist.data();
        qd.source = q.source;
        qd.r = q.r;
        qd.kb = kb;
        qd.header = reinterpret_cast<u64 *>(q.header);
        qd.header_words = 1024 / 8;
        qd.limit_ns = 0;
        order[i] = (u32)i;
    }
    std::stable_sort(order.begin(), order.end(), [&](u32 a, u32 b) {
        return (u64)qs[a].n + qs[a].m > (u64)qs[b].n + qs[b].m;
    });
    u32 next = 0;

    std::vector<Smem *> SS;
    std::vector<std::barrier<> *> bars;
    std::vector<WarpX *> wxs;
    for (int c = 0; c < P; c++) {
        Smem *S = (Smem *)aligned_alloc(64, (sizeof(Smem) + 63) / 64 * 64);
        memset(S, 0xCD, sizeof(Smem));
        SS.push_back(S);
        bars.push_back(new std::barrier<>(NT));
        WarpX *wx = new WarpX[NT / 32];
        for (int i = 0; i < NT / 32; i++) wx[i].bar = new std::barrier<>(32);
        wxs.push_back(wx);
    }
    std::vector<std::barrier<> *> cbars;
    if (C > 1) {
        g_cluster_size = C;
        for (int c = 0; c < P; c++) g_cta_smem[c] = SS[c];
        for (int k = 0; k < P / C; k++) cbars.push_back(new std::barrier<>(C * NT));
    }
    std::thread watchdog([&] {
        unsigned long long last = 0;
        for (int still = 0;;) {
            std::this_thread::sleep_for(std::chrono::seconds(1));
            const unsigned long long now = g_progress.load();
            if (now != last) {
                still = 0;
                last = now;
            } else if (++still == 30) {
                fprintf(stderr, "STALL: claimed %u of %llu; threads' last barrier lines:", next,
                        (unsigned long long)nq);
                for (int i = 0; i < NT * P; i += 32) fprintf(stderr, " %d", g_site_line[i]);
                fprintf(stderr, "\n");
                fflush(stderr);
                _exit(7);
            }
        }
    });
    watchdog.detach();
    const u32 nqu = (u32)nq;
    std::vector<std::thread> th;
    for (int c = 0; c < P; c++)
        for (int i = 0; i < NT; i++) {
            th.emplace_back([&, c, i] {
                threadIdx.x = i;
                blockIdx.x = c;
                g_gid = c * NT + i;
                g_cta_bar = bars[c];
                g_wx = wxs[c];
                Smem &S = *SS[c];
                if (C > 1) {
                    // the body of k_sssp_batch_cluster
                    g_cluster_bar = cbars[c / C];
                    const u32 rank = cluster_rank();
                    for (;;) {
                        if (rank == 0 && threadIdx.x == 0) S.bc[0] = atomicAdd(&next, 1u);
                        cluster_barrier();
                        const u32 qi = (u32)(rank == 0 ? S.bc[0] : dsmem_ld_u64(&S.bc[0], 0));
                        cluster_barrier();
                        if (qi >= nqu) break;
                        const QueryDesc &q = desc[order[qi]];
                        if (rank == 0)
                            for (u64 k = threadIdx.x; k < q.header_words; k += NT) q.header[k] = 0;
                        if (threadIdx.x == 0) g_err_sink_set(q.sc.err);
                        cluster_barrier();
                        state_load(S, q.hs);
                        ClusterTeam t{q.sc};
                        const Graph g = q.g;
                        run_query(t, S, g, q.source, q.dist, q.r, q.kb, q.limit_ns);
                        cluster_barrier();
                    }
                    return;
                }
                // the body of k_sssp_batch
                for (;;) {
                    if (threadIdx.x == 0) S.bc[0] = atomicAdd(&next, 1u);
                    __syncthreads();
                    const u32 qi = (u32)S.bc[0];
                    __syncthreads();
                    if (qi >= nqu) break;
                    const QueryDesc &q = desc[order[qi]];
                    for (u64 k = threadIdx.x; k < q.header_words; k += NT) q.header[k] = 0;
                    if (threadIdx.x == 0) g_err_sink_set(q.sc.err);
                    __syncthreads();
                    state_load(S, q.hs);
                    CtaTeam t{q.sc};
                    const Graph g = q.g;
                    run_query(t, S, g, q.source, q.dist, q.r, q.kb, q.limit_ns);
                    __syncthreads();
                }
            });
        }
    for (auto &x : th) x.join();
    FILE *o = fopen(argv[2], "wb");
    int rc = 0;
    for (auto &q : qs) {
        const u32 *err = q.p.sc.err;
        const u64 rec[3] = {err[0], q.p.sc.stats[STAT_ROUNDS], q.p.sc.stats[STAT_LEVELS]};
        fwrite(rec, 8, 3, o);
        fwrite(q.dist.data(), 8, q.n, o);
        if (err[0]) rc = 5;
    }
    fclose(o);
    return rc;
}
