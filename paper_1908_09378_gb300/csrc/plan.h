// plan.h -- host-side layout of a heap in one device workspace: the
// header (counters, status, barrier), team scratch, the BulkUpdate staging
// buffers and the ping-pong buffers of every level (Section 2.2 capacities).
// Host code only; included by pbh.cu.
#pragma once
#include <algorithm>
#include <cstddef>
#include <cstdint>

#include "core.cuh"
#include "concurrent.cuh"

namespace pbhk {

constexpr size_t ALIGN = 256;
constexpr u64 MAXGRID = 4096;
constexpr size_t HDR_BYTES = 4096;
// header offsets (bytes)
constexpr size_t OFF_STATS = 0;      // STAT_N u64
constexpr size_t OFF_ERR = 512;      // u32
constexpr size_t OFF_BAR = 576;      // u64
constexpr size_t OFF_UCOUNT = 640;   // u64
constexpr size_t OFF_CNT = 704;      // HeapCounters
constexpr size_t OFF_RES = 768;      // 16 u64
constexpr size_t OFF_BAR_A = 896;    // u64: barrier of the operation group (concurrent resolution)
constexpr size_t OFF_BAR_B = 904;    // u64: barrier of the deep group
constexpr size_t OFF_UCOUNT_B = 912; // u64
constexpr size_t OFF_RES_B = 920;    // 4 u64
constexpr size_t OFF_DEEP = 960;     // DeepSync
constexpr size_t OFF_HS = 1024;      // HeapState
constexpr u32 OPS_MAX = 4096;        // operations per launch of a sequence
static_assert(OFF_DEEP + sizeof(DeepSync) <= OFF_HS, "header");
static_assert(OFF_HS + sizeof(HeapState) <= HDR_BYTES, "header");
static_assert(STAT_N * 8 <= OFF_ERR, "stats");
static_assert((STAT_PROBE0 + STAT_NPROBES) * 8 <= OFF_ERR, "tracing slots");

inline size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

inline u32 levels_for(u64 capacity, u64 d)
{
    u32 q = 1;
    u64 span = d; // d * 4^(q-1)
    while (span < capacity && q < (u32)MAXQ) {
        span *= 4;
        q++;
    }
    return q;
}

// Lay out one heap (header, scratch, U buffers, levels) from `base`; with
// base == nullptr only the size is computed.  `cur_in` is the validity array
// (nullptr: reserve key_space words for it in the workspace).
struct Plan {
    size_t bytes = 0;
    HeapState hs{};
    Scratch sc{};
    Scratch sc2{};         // the deep group's scratch (heaps that run operation sequences)
    OpDesc *ops = nullptr; // OPS_MAX operation descriptors (same)
    u32 *seen = nullptr;   // two key_space-bit maps for pbh_validate (heap API)
    u64 *cur = nullptr;
    u64 key_space = 0;
};

// `take(bytes)` hands out the memory of each buffer in turn; `hdr` is the
// header block (nullptr when only sizing).
template <class Take>
bool plan_heap_with(Take &&take, char *hdr, u64 key_space, u64 d, u64 capacity, u64 *cur_in, u64 grid_ctas,
                    Plan *out, bool groups = false)
{
    if (d == 0 || key_space == 0) return false;
    if (capacity == 0) capacity = key_space;
    const u32 q = levels_for(capacity, d);
    if (q >= (u32)MAXQ) return false;
    char *base = hdr;
    Plan p;
    HeapState &hs = p.hs;
    hs.q = q;
    hs.d = d;
    hs.key_space = key_space;
    // largest merge: Empty at the last level
    u64 maxel = 0;
    u64 pw = 1;
    for (u32 i = 0; i < q; i++, pw *= 4) maxel = std::max(maxel, 4 * d * pw);
    const u64 max_tiles = maxel / TILE + 2;
    p.sc.stats = base ? reinterpret_cast<u64 *>(base + OFF_STATS) : nullptr;
    p.sc.err = base ? reinterpret_cast<u32 *>(base + OFF_ERR) : nullptr;
    p.sc.bar = base ? reinterpret_cast<u64 *>(base + OFF_BAR) : nullptr;
    p.sc.ucount = base ? reinterpret_cast<u64 *>(base + OFF_UCOUNT) : nullptr;
    p.sc.res = base ? reinterpret_cast<u64 *>(base + OFF_RES) : nullptr;
    const bool grid = grid_ctas > 1;
    p.sc.partials = reinterpret_cast<u64 *>(take(8 * std::max<u64>(grid_ctas, 1)));
    p.sc.splits = reinterpret_cast<u64 *>(take(grid ? 8 * (max_tiles + 2) : 8));
    p.sc.bits = reinterpret_cast<unsigned char *>(take(grid ? (max_tiles + 2) * NT : 8));
    if (groups) {
        // a second set of merge scratch for the deep group, and the operations
        p.sc2 = p.sc;
        p.sc2.bar = base ? reinterpret_cast<u64 *>(base + OFF_BAR_B) : nullptr;
        p.sc2.ucount = base ? reinterpret_cast<u64 *>(base + OFF_UCOUNT_B) : nullptr;
        p.sc2.res = base ? reinterpret_cast<u64 *>(base + OFF_RES_B) : nullptr;
        p.sc2.partials = reinterpret_cast<u64 *>(take(8 * std::max<u64>(grid_ctas, 1)));
        p.sc2.splits = reinterpret_cast<u64 *>(take(8 * (max_tiles + 2)));
        p.sc2.bits = reinterpret_cast<unsigned char *>(take((max_tiles + 2) * NT));
        p.ops = reinterpret_cast<OpDesc *>(take(sizeof(OpDesc) * OPS_MAX));
        p.seen = reinterpret_cast<u32 *>(take(2 * 4 * ((key_space + 31) / 32)));
    }
    if (cur_in) {
        // SSSP: the validity array is the caller's distance array; one round
        // tag per vertex dedups each round's BulkUpdate batch
        hs.cur = cur_in;
        hs.mark = reinterpret_cast<u32 *>(take(4 * key_space));
    } else {
        hs.cur = reinterpret_cast<u64 *>(take(8 * key_space));
    }
    hs.U[0] = reinterpret_cast<u64 *>(take(8 * d));
    hs.U[1] = reinterpret_cast<u64 *>(take(8 * d));
    pw = 1;
    for (u32 i = 0; i < q; i++, pw *= 4) {
        Level &L = hs.L[i];
        L.capB = 2 * d * pw;
        L.capS = d * pw;
        L.bufB = 4 * d * pw;
        L.bufS = i == 0 ? d : 2 * d * pw;
        L.B[0] = reinterpret_cast<u64 *>(take(8 * L.bufB));
        L.B[1] = reinterpret_cast<u64 *>(take(8 * L.bufB));
        if (i == 0) {
            L.S[0] = hs.U[0];
            L.S[1] = hs.U[1];
        } else {
            L.S[0] = reinterpret_cast<u64 *>(take(8 * L.bufS));
            L.S[1] = reinterpret_cast<u64 *>(take(8 * L.bufS));
        }
        L.T = INF;
    }
    p.cur = hs.cur;
    p.key_space = key_space;
    *out = p;
    return true;
}

// Bump layout inside one workspace starting at `base` (header first); with
// base == nullptr only the size is computed.
inline bool plan_heap(char *base, u64 key_space, u64 d, u64 capacity, u64 *cur_in, u64 grid_ctas, Plan *out,
                      bool groups = false)
{
    size_t off = HDR_BYTES;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes);
        return base ? base + o : nullptr;
    };
    if (!plan_heap_with(take, base, key_space, d, capacity, cur_in, grid_ctas, out, groups)) return false;
    out->bytes = off;
    return true;
}

inline u32 key_bits(u32 n)
{
    u32 kb = 1;
    while (kb < 32 && (1ull << kb) < n) kb++;
    return kb;
}

} // namespace pbhk
