// One parDijkstra query (run_query of core.cuh) on P emulated CTAs joined by
// the grid-team barrier, or (TEAM = 1) forming one thread-block cluster
// joined by the cluster barrier (ClusterTeam, the body of k_sssp_cluster),
// for the CPU tests.  STALL = 1: CTA 0 withholds one grid-barrier arrival
// and every barrier wait is bounded by 200 ms; LIMIT_MS: the query's time
// limit (0 = the default).  Usage:
//   harness GRAPH OUT P SETTLE [TEAM [STALL [LIMIT_MS]]]
// GRAPH: u64 n, m, source, r, d; u64 row_ptr[n+1]; u32 col[m]; u32 w[m].
// OUT receives the n distances (u64).  Prints the latched status, site,
// rounds and levels on stderr; exits 0 (ok), 5 (latched device error) or 7
// (no thread made progress for 30 s: the emulated kernel is stuck).
// Every buffer is its own allocation, so a sanitizer sees any overrun.
#include "cuda_shim.h"
#include "core_host.h"
#include "plan_host.h"
#include <vector>
using namespace pbhk;

int main(int argc, char **argv)
{
    if (argc < 5) return 1;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    uint64_t hdr[5];
    if (fread(hdr, 8, 5, f) != 5) return 2;
    const u32 n = (u32)hdr[0];
    const u64 m = hdr[1];
    const u32 source = (u32)hdr[2], r = (u32)hdr[3], d = (u32)hdr[4];
    u64 *row_ptr = (u64 *)malloc(8 * (n + 1));
    u32 *col = (u32 *)malloc(4 * m + 4);
    u32 *w = (u32 *)malloc(4 * m + 4);
    if (fread(row_ptr, 8, n + 1, f) != n + 1 || fread(col, 4, m, f) != m || fread(w, 4, m, f) != m) return 3;
    fclose(f);
    const int P = atoi(argv[3]);
    if (P < 2 || P > 16) return 1;
    const bool cluster = argc > 5 && atoi(argv[5]) == 1;
    const bool stall = argc > 6 && atoi(argv[6]) == 1;
    const u64 limit_ns = argc > 7 ? 1000000ull * strtoull(argv[7], nullptr, 10) : 0;
    u64 *Dist = (u64 *)malloc(8ull * n);
    char *header = (char *)calloc(HDR_BYTES, 1);
    std::vector<void *> bufs;
    auto take = [&](size_t bytes) {
        void *p = malloc(bytes ? bytes : 8);
        memset(p, 0xAB, bytes);
        bufs.push_back(p);
        return (char *)p;
    };
    Plan p;
    gridDim.x = P;
    if (!plan_heap_with(take, header, n, d, n, Dist, P, &p)) return 4;
    const u32 kb = key_bits(n);
    p.hs.reset_on_extract = 0;
    p.hs.keymask = (1ull << kb) - 1;
    p.hs.settle = atoi(argv[4]) ? 1 : 0;
    if (stall) {
        p.sc.stall = 1;
        p.sc.wait_ns = 200000000ull;
    }
    Graph g{n, m, row_ptr, col, w};

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
    std::barrier<> cluster_bar(P * NT);
    if (cluster) {
        g_cluster_size = P;
        for (int c = 0; c < P; c++) g_cta_smem[c] = SS[c];
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
                fprintf(stderr, "STALL: status %u site %u; threads' last barrier lines:", p.sc.err[0], p.sc.err[1]);
                for (int i = 0; i < NT * P; i += 32) fprintf(stderr, " %d", g_site_line[i]);
                fprintf(stderr, "\n");
                fflush(stderr);
                _exit(7);
            }
        }
    });
    watchdog.detach();
    std::vector<std::thread> th;
    for (int c = 0; c < P; c++)
        for (int i = 0; i < NT; i++) {
            th.emplace_back([&, c, i] {
                threadIdx.x = i;
                blockIdx.x = c;
                g_gid = c * NT + i;
                g_cta_bar = bars[c];
                g_wx = wxs[c];
                Smem *S = SS[c];
                const u64 *src = reinterpret_cast<const u64 *>(&p.hs);
                u64 *dst = reinterpret_cast<u64 *>(&S->hs);
                for (u32 k = i; k < sizeof(HeapState) / 8; k += NT) dst[k] = src[k];
                if (cluster) {
                    g_cluster_bar = &cluster_bar;
                    if (i == 0) g_err_sink_set(p.sc.err);
                    __syncthreads();
                    ClusterTeam t{p.sc};
                    run_query(t, *S, g, source, Dist, r, kb, limit_ns);
                } else {
                    if (i == 0) g_err_sink_set(p.sc.err, p.sc.bar);
                    __syncthreads();
                    GridTeam t{p.sc};
                    run_query(t, *S, g, source, Dist, r, kb, limit_ns);
                }
            });
        }
    for (auto &x : th) x.join();
    const u32 *err = p.sc.err;
    fprintf(stderr, "status %u site %u rounds %llu levels %llu settled %llu\n", err[0], err[1],
            (unsigned long long)p.sc.stats[STAT_ROUNDS], (unsigned long long)p.sc.stats[STAT_LEVELS],
            (unsigned long long)p.sc.stats[STAT_SETTLED]);
    FILE *o = fopen(argv[2], "wb");
    fwrite(Dist, 8, n, o);
    fclose(o);
    return err[0] ? 5 : 0;
}
