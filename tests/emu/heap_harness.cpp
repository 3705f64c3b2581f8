// A stream of heap-API operations (heap_op of heapop.cuh) on P emulated CTAs
// joined by the grid-team barrier, each followed by the debug validator
// (heap_validate) on CTA 0, for the CPU tests.  Usage:
//   heap_harness OPS OUT P
// OPS: u64 key_space, d, nops; per operation u64 kind, count, r, then
// u32 keys[count], u32 prios[count] (kind: 0 BulkUpdate, 1 extract,
// 2 delete, 3 assign; r for extract).
// OUT, per operation: u64 nout, u32 keys[nout], u32 prios[nout] (extract
// only; nout = 0 otherwise), then u64 violations, stored, valid keys, live
// (the counters' inserted - extracted - deleted).
// Exits 0 (ok), 5 (latched device error) or 7 (no thread made progress for
// 30 s: the emulated kernel is stuck).
#include "cuda_shim.h"
#include "core_host.h"
#include "heapop_host.h"
#include "plan_host.h"
#include <vector>
using namespace pbhk;

struct Op {
    u64 kind, count, r;
    std::vector<u32> keys, prios;
};

int main(int argc, char **argv)
{
    if (argc < 4) return 1;
    FILE *f = fopen(argv[1], "rb");
    if (!f) return 2;
    uint64_t hdr[3];
    if (fread(hdr, 8, 3, f) != 3) return 2;
    const u64 key_space = hdr[0], d = hdr[1], nops = hdr[2];
    std::vector<Op> ops(nops);
    for (auto &o : ops) {
        uint64_t h[3];
        if (fread(h, 8, 3, f) != 3) return 3;
        o.kind = h[0];
        o.count = h[1];
        o.r = h[2];
        o.keys.resize(o.count + 1);
        o.prios.resize(o.count + 1);
        if (fread(o.keys.data(), 4, o.count, f) != o.count || fread(o.prios.data(), 4, o.count, f) != o.count)
            return 3;
    }
    fclose(f);
    const int P = atoi(argv[3]);
    if (P < 2 || P > 512) return 1;
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
    if (!plan_heap_with(take, header, key_space, d, key_space, nullptr, P, &p, true)) return 4;
    p.hs.reset_on_extract = 1;
    p.hs.keymask = 0xffffffffull;
    for (u64 k = 0; k < key_space; k++) p.cur[k] = INF;
    HeapState *g_hs = reinterpret_cast<HeapState *>(header + OFF_HS);
    memcpy(g_hs, &p.hs, sizeof(HeapState));
    HeapCounters *cnt = reinterpret_cast<HeapCounters *>(header + OFF_CNT);
    const u64 words = (key_space + 31) / 32;
    u32 *seen = p.seen, *dup = p.seen + words;
    std::vector<u32> kout(d + 1), pout(d + 1);
    u32 nout = 0;
    u64 vres[3];
    FILE *o = fopen(argv[2], "wb");

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
    std::barrier<> launch(P * NT); // the boundary between two kernel launches
    std::thread watchdog([&] {
        unsigned long long last = 0;
        for (int still = 0;;) {
            std::this_thread::sleep_for(std::chrono::seconds(1));
            const unsigned long long now = g_progress.load();
            if (now != last) {
                still = 0;
                last = now;
            } else if (++still == 30) {
                fprintf(stderr, "STALL: status %u site %u\n", p.sc.err[0], p.sc.err[1]);
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
                for (u64 k = 0; k < nops; k++) {
                    const Op &op = ops[k];
                    static const int kinds[4] = {OP_BULK, OP_EXTRACT, OP_DELETE, OP_ASSIGN};
                    GridTeam t{p.sc};
                    t.init();
                    if (i == 0) g_err_sink_set(p.sc.err, p.sc.bar);
                    heap_op(t, *S, g_hs, cnt, kinds[op.kind], op.keys.data(), op.prios.data(), (u32)op.count,
                            (u32)op.r, kout.data(), pout.data(), &nout);
                    launch.arrive_and_wait();
                    if (c == 0) {
                        if (i == 0) {
                            memset(seen, 0, 2 * 4 * words);
                            memset(vres, 0, sizeof(vres));
                            g_err_sink_set(nullptr);
                        }
                        __syncthreads();
                        heap_validate(*S, g_hs, reinterpret_cast<u32 *>(vres), vres + 1, vres + 2, seen, dup);
                    }
                    launch.arrive_and_wait();
                    if (c == 0 && i == 0) {
                        const u64 n = op.kind == 1 ? nout : 0;
                        fwrite(&n, 8, 1, o);
                        fwrite(kout.data(), 4, n, o);
                        fwrite(pout.data(), 4, n, o);
                        const u64 live = cnt->inserted - cnt->extracted - cnt->deleted;
                        const u64 rec[4] = {vres[0] & 0xffffffffull, vres[1], vres[2], live};
                        fwrite(rec, 8, 4, o);
                        nout = 0;
                    }
                    launch.arrive_and_wait();
                }
            });
        }
    for (auto &x : th) x.join();
    fclose(o);
    const u32 *err = p.sc.err;
    fprintf(stderr, "status %u site %u levels %u\n", err[0], err[1], p.hs.q);
    return err[0] ? 5 : 0;
}
