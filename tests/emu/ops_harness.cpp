// A sequence of heap operations in one emulated cooperative launch with
// concurrent resolution of non-adjacent levels (run_ops and deep_serve of
// concurrent.cuh): CTAs [0, nA) are the operation group, [nA, P) the deep
// group, as in k_pbh_ops.  Then the debug validator (heap_validate) on CTA 0.
// For the CPU tests.  Usage:
//   ops_harness OPS OUT P nA
// OPS: u64 key_space, d, nops; per operation u64 kind, count, r, then
// u32 keys[count], u32 prios[count] (kind: 0 BulkUpdate, 1 extract).
// OUT: per operation u64 nout, u32 keys[nout], u32 prios[nout] (nout = 0 for
// a BulkUpdate); then u64 violations, stored, valid keys, live, status, and
// the resolve count of every level (u64 q, then q counts).
// Exits 0 (ok), 5 (latched device error) or 7 (no thread made progress for
// 30 s: the emulated kernel is stuck).
#include "cuda_shim.h"
#include "core_host.h"
#include "concurrent_host.h"
#include "heapop_host.h"
#include "plan_host.h"
#include <vector>
using namespace pbhk;

struct Op {
    u64 kind, count, r;
    std::vector<u32> keys, prios, kout, pout;
    u32 nout = 0;
};

int main(int argc, char **argv)
{
    if (argc < 5) return 1;
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
        if (o.kind > 1 || o.count > d || o.r > d) return 3;
        o.keys.resize(o.count + 1);
        o.prios.resize(o.count + 1);
        o.kout.resize(o.r + 1);
        o.pout.resize(o.r + 1);
        if (fread(o.keys.data(), 4, o.count, f) != o.count || fread(o.prios.data(), 4, o.count, f) != o.count)
            return 3;
    }
    fclose(f);
    const int P = atoi(argv[3]);
    const u32 nA = (u32)atoi(argv[4]);
    if (P < 2 || P > 64 || nA < 1 || nA > (u32)P) return 1;
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
    DeepSync *ds = reinterpret_cast<DeepSync *>(header + OFF_DEEP);
    Scratch scA = p.sc;
    scA.bar = reinterpret_cast<u64 *>(header + OFF_BAR_A);
    Scratch scB = p.sc2;

    // the descriptors, as pbh_run_ops copies them to the device
    std::vector<OpDesc> descs(nops);
    for (u64 k = 0; k < nops; k++) {
        Op &o = ops[k];
        descs[k] = OpDesc{o.kind == 0 ? (u32)OP_BULK : (u32)OP_EXTRACT, (u32)o.count, (u32)o.r, 0, o.keys.data(),
                          o.prios.data(), o.kout.data(), o.pout.data(), &o.nout};
    }
    const u64 words = (key_space + 31) / 32;
    u32 *seen = p.seen, *dup = p.seen + words;
    u64 vres[3] = {0, 0, 0};

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
    std::barrier<> launch(P * NT); // the end of the cooperative launch
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
                Smem &S = *SS[c];
                // the body of k_pbh_ops
                const bool op_group = (u32)c < nA;
                GroupTeam t{op_group ? scA : scB, op_group ? 0u : nA, op_group ? nA : (u32)P - nA};
                t.init();
                if (i == 0) g_err_sink_set(t.sc.err, t.sc.bar);
                state_load(S, g_hs);
                const bool deep = S.hs.q > 2 && nA < (u32)P;
                if (op_group) {
                    OpsCtl ctl{g_hs, ds, 0, deep, true, true, false};
                    run_ops(t, S, cnt, descs.data(), (u32)nops, ctl);
                } else if (deep) {
                    deep_serve(t, S, g_hs, ds);
                }
                launch.arrive_and_wait();
                if (c == 0) {
                    if (i == 0) {
                        memset(seen, 0, 2 * 4 * words);
                        g_err_sink_set(nullptr);
                    }
                    __syncthreads();
                    heap_validate(S, g_hs, reinterpret_cast<u32 *>(vres), vres + 1, vres + 2, seen, dup);
                }
            });
        }
    for (auto &x : th) x.join();
    FILE *o = fopen(argv[2], "wb");
    for (const Op &op : ops) {
        const u64 n = op.kind == 1 ? op.nout : 0;
        fwrite(&n, 8, 1, o);
        fwrite(op.kout.data(), 4, n, o);
        fwrite(op.pout.data(), 4, n, o);
    }
    const u32 *err = p.sc.err;
    const u64 live = cnt->inserted - cnt->extracted - cnt->deleted;
    const u64 rec[5] = {vres[0] & 0xffffffffull, vres[1], vres[2], live, err[0]};
    fwrite(rec, 8, 5, o);
    const u64 q = g_hs->q;
    fwrite(&q, 8, 1, o);
    for (u64 i = 0; i < q; i++) fwrite(&g_hs->L[i].nres, 8, 1, o);
    fclose(o);
    fprintf(stderr, "status %u site %u levels %u\n", err[0], err[1], g_hs->q);
    return err[0] ? 5 : 0;
}
