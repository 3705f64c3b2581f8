// The continuous-batching server on the CPU: the body of k_serve on P
// emulated CTAs, taking requests from a ring of SLOTS records that a host
// thread fills as srv_submit does (the record, then the tail), reusing a
// slot only once its completion flag reports the request before; then the
// stop word.  Each request is one parDijkstra query on its own heap
// (CtaTeam); or, with a cluster size C >= 2, the body of k_serve_cluster:
// P / C clusters, whose first CTA claims and waits for a request and the
// others read the claim through distributed shared memory, each request on
// one cluster (ClusterTeam).  For the CPU tests.  Usage:
//   serve_harness QUERIES OUT P SLOTS [C]
// QUERIES: as batch_harness (u64 nq; per query u64 n, m, source, r, d;
// u64 row_ptr[n+1]; u32 col[m]; u32 w[m]).
// OUT: per request u64 status, u64 done flag, then u64 dist[n].
// Exits 0 (ok), 5 (a request latched a device error, or the server its
// status) or 7 (no thread made progress for 30 s: the emulation is stuck).
#include "cuda_shim.h"
#include "core_host.h"
#include "kernels_host.h"
#include "plan_host.h"
#include <vector>
using namespace pbhk;

struct Query {
    u32 n, source, r, d;
    u64 m;
    std::vector<u64> row_ptr, dist;
    std::vector<u32> col, w;
    Plan p;
    char *header = nullptr;
};

int main(int argc, char **argv)
{
    if (argc < 5) return 1;
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
    const u32 slots = (u32)atoi(argv[4]);
    const int C = argc > 5 ? atoi(argv[5]) : 1;
    if (P < 1 || P > 16 || slots < 1 || C < 1 || P % C) return 1;
    gridDim.x = P;
    std::vector<void *> bufs;
    auto take = [&](size_t bytes) {
        void *p = malloc(bytes ? bytes : 8);
        memset(p, 0xAB, bytes);
        bufs.push_back(p);
        return (char *)p;
    };
    std::vector<ServeRecord> ring(slots);
    memset(ring.data(), 0, sizeof(ServeRecord) * slots);
    ServeCtl ctl;
    memset(&ctl, 0, sizeof(ctl));
    std::vector<u64> done(slots, 0), t_begin(slots, 0), t_end(slots, 0), flag(nq, 0);
    u64 head = 0;

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
    // the wait for a published request (thread 0 of the claiming CTA); the
    // kernel's volatile loads of the mapped control words are acquire loads
    // here, as the host thread's stores are atomic
    auto mapped = [](u64 &w) { return std::atomic_ref<u64>(w).load(std::memory_order_acquire); };
    auto claim = [&](Smem &S) {
        const u64 idx = atomicAdd(&head, 1ull);
        u64 ok = 1;
        u64 t0 = gtimer(), seen = 0;
        for (u32 spin = 0; mapped(ctl.tail) <= idx; spin++) {
            if (std::atomic_ref<u32>(ctl.stop).load(std::memory_order_acquire)) {
                ok = 0;
                break;
            }
            if ((spin & 63) == 0) {
                const u64 now = gtimer();
                const u64 sign = mapped(ctl.heartbeat) + mapped(ctl.tail);
                if (sign != seen) {
                    seen = sign;
                    t0 = now;
                }
                const u64 idle_set = mapped(ctl.idle_ns);
                if (now - t0 > (idle_set ? idle_set : SERVE_IDLE_NS)) {
                    atomicCAS(&ctl.status, 0u, (u32)ST_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(1000);
        }
        __threadfence_system();
        S.bc[0] = idx;
        S.bc[1] = ok;
    };
    std::thread watchdog([&] {
        unsigned long long last = 0;
        for (int still = 0;;) {
            std::this_thread::sleep_for(std::chrono::seconds(1));
            const unsigned long long now = g_progress.load();
            if (now != last) {
                still = 0;
                last = now;
            } else if (++still == 30) {
                fprintf(stderr, "STALL: head %llu tail %llu\n", (unsigned long long)head,
                        (unsigned long long)ctl.tail);
                fflush(stderr);
                _exit(7);
            }
        }
    });
    watchdog.detach();

    // the host: srv_submit's steps for every request, then the stop word
    // once every request has completed
    std::thread host([&] {
        auto flag_of = [&](u32 slot) { return std::atomic_ref<u64>(done[slot]).load(std::memory_order_acquire); };
        for (u64 k = 0; k < nq; k++) {
            const u32 slot = (u32)(k % slots);
            while (k >= slots && flag_of(slot) != k - slots + 1) std::this_thread::yield();
            Query &q = qs[k];
            q.header = (char *)calloc(HDR_BYTES, 1);
            if (!plan_heap_with(take, q.header, q.n, q.d, q.n, q.dist.data(), C, &q.p)) _exit(4);
            const u32 kb = key_bits(q.n);
            q.p.hs.reset_on_extract = 0;
            q.p.hs.keymask = (1ull << kb) - 1;
            ServeRecord &rec = ring[slot];
            rec.hs = q.p.hs;
            QueryDesc qd{};
            qd.sc = q.p.sc;
            qd.hs = &rec.hs;
            qd.g = Graph{q.n, q.m, q.row_ptr.data(), q.col.data(), q.w.data()};
            qd.dist = q.dist.data();
            qd.source = q.source;
            qd.r = q.r;
            qd.kb = kb;
            qd.header = reinterpret_cast<u64 *>(q.header);
            qd.header_words = 1024 / 8;
            rec.q = qd;
            std::atomic_thread_fence(std::memory_order_seq_cst); // the record before the tail
            std::atomic_ref<u64>(ctl.tail).store(k + 1, std::memory_order_release);
            g_progress.fetch_add(1, std::memory_order_relaxed);
        }
        for (u64 k = nq > slots ? nq - slots : 0; k < nq; k++)
            while (flag_of((u32)(k % slots)) != k + 1) std::this_thread::yield();
        for (u64 k = 0; k < nq; k++) flag[k] = 1; // every request reported its completion in turn
        std::atomic_ref<u32>(ctl.stop).store(1, std::memory_order_release);
    });

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
                    // the body of k_serve_cluster
                    g_cluster_bar = cbars[c / C];
                    const u32 rank = cluster_rank();
                    for (;;) {
                        if (rank == 0 && threadIdx.x == 0) claim(S);
                        cluster_barrier();
                        const u64 idx = rank == 0 ? S.bc[0] : dsmem_ld_u64(&S.bc[0], 0);
                        const bool ok = (rank == 0 ? S.bc[1] : dsmem_ld_u64(&S.bc[1], 0)) != 0;
                        cluster_barrier();
                        if (!ok) break;
                        const u32 slot = (u32)(idx % slots);
                        const QueryDesc q = ring[slot].q;
                        if (rank == 0) {
                            if (threadIdx.x == 0) t_begin[slot] = gtimer();
                            for (u64 k = threadIdx.x; k < q.header_words; k += NT) q.header[k] = 0;
                        }
                        if (threadIdx.x == 0) g_err_sink_set(q.sc.err);
                        cluster_barrier();
                        state_load(S, q.hs);
                        ClusterTeam t{q.sc};
                        run_query(t, S, q.g, q.source, q.dist, q.r, q.kb, q.limit_ns);
                        cluster_barrier();
                        if (rank == 0 && threadIdx.x == 0) {
                            __threadfence_system();
                            t_end[slot] = gtimer();
                            std::atomic_ref<u64>(done[slot]).store(idx + 1, std::memory_order_release);
                        }
                    }
                    return;
                }
                // the body of k_serve
                for (;;) {
                    if (threadIdx.x == 0) claim(S);
                    __syncthreads();
                    const u64 idx = S.bc[0];
                    const bool ok = S.bc[1] != 0;
                    __syncthreads();
                    if (!ok) break;
                    const u32 slot = (u32)(idx % slots);
                    const ServeRecord &rec = ring[slot];
                    const QueryDesc q = rec.q;
                    if (threadIdx.x == 0) t_begin[slot] = gtimer();
                    for (u64 k = threadIdx.x; k < q.header_words; k += NT) q.header[k] = 0;
                    if (threadIdx.x == 0) g_err_sink_set(q.sc.err);
                    __syncthreads();
                    state_load(S, q.hs);
                    CtaTeam t{q.sc};
                    run_query(t, S, q.g, q.source, q.dist, q.r, q.kb, q.limit_ns);
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        __threadfence_system();
                        t_end[slot] = gtimer();
                        std::atomic_ref<u64>(done[slot]).store(idx + 1, std::memory_order_release);
                    }
                }
            });
        }
    for (auto &x : th) x.join();
    host.join();
    FILE *o = fopen(argv[2], "wb");
    int rc = ctl.status ? 5 : 0;
    for (auto &q : qs) {
        const u32 *err = q.p.sc.err;
        const u64 rec[2] = {err[0], flag[&q - qs.data()]};
        fwrite(rec, 8, 2, o);
        fwrite(q.dist.data(), 8, q.n, o);
        if (err[0]) rc = 5;
    }
    fclose(o);
    return rc;
}
