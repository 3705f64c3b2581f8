// concurrent.cuh -- concurrent resolution of non-adjacent levels (Section
// 2.2.1, Figure 2, Theorem 3): a sequence of heap operations in one launch
// whose CTAs form two groups.
//
//   * The operation group runs the operations (BulkUpdate, extract), every
//     Resolve(0) and every Resolve(1).
//   * The deep group runs every Resolve(2) and the deeper resolves it
//     triggers (Resolve(i) after every fourth Resolve(i-1)).
//
// Resolve(2) number k may start once Resolve(1) number 4k has finished, and
// must finish before Resolve(1) number 4k+1 starts (the order
// Res_{i-1}(4k) -> Res_i(k) -> Res_{i-1}(4k+1) of Figure 2).  In between, the
// operation group keeps running operations and their Resolve(0), which touch
// levels 0 and 1 only, while the deep group works on levels 2 and deeper:
// non-adjacent levels resolve at the same time.  Three monotone counters
// carry the order: `ready` (released by the operation group after Resolve(1)
// number 4k: Resolve(2) number k may start), `done` (released by the deep
// group when Resolve(2) number k has finished: level 2 is the operation
// group's again) and `idle` (released when the deeper resolves that
// Resolve(2) number k triggered have finished too).  So Resolve(3) and deeper
// overlap the operation group's next Resolve(1) as well, which touches levels
// 1 and 2 only.  The levels' state (run heads, lengths, thresholds, resolve
// counts) is handed over through the heap state in global memory: level 2
// at `ready` and `done`; levels 3 and deeper belong to the deep group, and
// the operation group takes them only after `idle` (the fill cascade of an
// extract that finds B_0 short, a signal buffer pushed over capacity), and
// hands them back, marked changed, with its next `ready`.  Every cross-group
// wait is bounded.
//
// Each group is a team with its own barrier counter and merge scratch; the
// status word and the counters are shared.
#pragma once
#include "core.cuh"

namespace pbhk {

// The words through which the two groups hand the deep levels over.
struct DeepSync {
    u64 ready; // Resolve(2) calls the operation group has released (monotone)
    u64 done;  // Resolve(2) calls the deep group has finished
    u64 idle;  // ... with the deeper resolves they triggered
    u32 stop;  // the operation group has finished: the deep group leaves
    u32 dirty; // the `ready` with which the operation group handed back levels 3 and deeper, changed
};

// One heap operation of a sequence (the kind values are OP_BULK, OP_EXTRACT).
struct OpDesc {
    u32 kind, count, r, pad;
    const u32 *keys, *prios;
    u32 *kout, *pout, *nout;
};

// A team of the CTAs [first, first + count) of a cooperative launch, joined
// by a bounded software barrier on its own counter sc.bar.
struct GroupTeam {
    static constexpr bool kSingle = false;
    static constexpr bool kTimed = true;
    static constexpr bool kSoftBarrier = true;
    __device__ __forceinline__ bool failed() const { return s_err_flag != 0; }
    Scratch sc;
    u32 first, count;
    u64 gen = 0;
    u64 nsync = 0;
    bool withhold = false;
    __device__ __forceinline__ u32 ncta() const { return count; }
    __device__ __forceinline__ u32 cta() const { return blockIdx.x - first; }
    __device__ void init()
    {
        if (threadIdx.x == 0) gen = ld_acquire(sc.bar) / count;
    }
    __device__ __forceinline__ void sync() { GridTeam::soft_barrier(sc, count, gen, nsync, withhold); }
};

__device__ __forceinline__ void st_release(u64 *p, u64 v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Copy levels [from, to) of the heap state (to = 0: up to q) between global
// and shared memory.
__device__ __forceinline__ u32 level_words(const Smem &S, int from, int to)
{
    static_assert(sizeof(Level) % 8 == 0, "levels are copied as words");
    const int end = to ? min(to, (int)S.hs.q) : (int)S.hs.q;
    return end > from ? (u32)((end - from) * sizeof(Level) / 8) : 0;
}

__device__ __forceinline__ void levels_load(Smem &S, const HeapState *g, int from, int to = 0)
{
    const u64 *src = reinterpret_cast<const u64 *>(&g->L[from]);
    u64 *dst = reinterpret_cast<u64 *>(&S.hs.L[from]);
    const u32 words = level_words(S, from, to);
    for (u32 i = threadIdx.x; i < words; i += NT) dst[i] = ldg_cg(src + i);
    __syncthreads();
}

__device__ __forceinline__ void levels_store(const Smem &S, HeapState *g, int from, int to = 0)
{
    const u64 *src = reinterpret_cast<const u64 *>(&S.hs.L[from]);
    u64 *dst = reinterpret_cast<u64 *>(&g->L[from]);
    const u32 words = level_words(S, from, to);
    for (u32 i = threadIdx.x; i < words; i += NT) dst[i] = src[i];
}

// The operation group's side of the hand-over.  It owns level 2 from the
// start until it releases a Resolve(2), and again once the deep group has
// finished it (`done`); it owns levels 3 and deeper only after the deep group
// has finished everything released (`idle`), until its next release.  While
// it owns levels, its shared-memory copy of their state is the current one.
struct OpsCtl {
    HeapState *g_hs;
    DeepSync *ds;
    u64 ready_pub; // Resolve(2) calls released so far (the same in every thread)
    bool deep;     // a deep group exists and the heap has levels 2 and deeper
    bool own2;     // the operation group owns level 2 now
    bool own_all;  // ... and levels 3 and deeper
    bool dirty;    // it changed levels 3 and deeper since it took them
};

// Wait (bounded) until the counter *w reaches upto.
template <class Team>
__device__ void deep_wait(Team &t, const u64 *w, u64 upto)
{
    if (threadIdx.x == 0) {
        u64 t0 = 0;
        for (u32 spins = 0; ld_acquire(w) < upto; spins++) {
            if ((spins & 255) == 0) {
                if (read_err(t.sc.err) != 0) {
                    s_err_flag = 1;
                    break;
                }
                const u64 now = gtimer();
                if (t0 == 0) {
                    t0 = now;
                } else if (now - t0 > SPIN_NS) {
                    raise_err(t.sc.err, ST_TIMEOUT, 30);
                    break;
                }
            }
        }
    }
    __syncthreads();
}

// Take level 2 back: wait until the last Resolve(2) released has finished,
// then reload its state.
template <class Team>
__device__ void own_level2(Team &t, Smem &S, OpsCtl &c)
{
    if (c.own2) return;
    deep_wait(t, &c.ds->done, c.ready_pub);
    levels_load(S, c.g_hs, 2, 3);
    c.own2 = true;
}

// Take every deep level back: wait until the deep group is idle, then
// reload their state.
template <class Team>
__device__ void own_all_levels(Team &t, Smem &S, OpsCtl &c)
{
    if (c.own_all) return;
    deep_wait(t, &c.ds->idle, c.ready_pub);
    levels_load(S, c.g_hs, c.own2 ? 3 : 2);
    c.own2 = c.own_all = true;
}

// Release Resolve(2) number `ready` to the deep group, after a team barrier
// (every CTA's merges complete): CTA 0 writes level 2's state (and that of
// the deeper levels, if the operation group changed them) to global memory,
// then releases the count.  Ends with a team barrier.
template <class Team>
__device__ void deep_release(Team &t, Smem &S, OpsCtl &c, u64 ready)
{
    if (t.cta() == 0) {
        levels_store(S, c.g_hs, 2, c.dirty ? 0 : 3);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (c.dirty) *(volatile u32 *)&c.ds->dirty = (u32)ready;
            st_release(&c.ds->ready, ready);
        }
    }
    c.ready_pub = ready;
    c.own2 = c.own_all = c.dirty = false;
    t.sync();
}

// Empty level i ≥ 1 and the signal buffers it pushes over capacity, on the
// operation group: a cascade past level 2 needs the deeper levels.
template <class Team>
__device__ void conc_empty_cascade(Team &t, Smem &S, OpsCtl &c, int i)
{
    HeapState &hs = S.hs;
    for (int j = i; j < (int)hs.q && !t.failed(); j++) {
        if (j > i && hs.L[j].slen <= hs.L[j].capS) break;
        if (c.deep && j >= 2) {
            own_all_levels(t, S, c);
            c.dirty = true;
        }
        empty_level_once(t, S, j);
    }
}

// The schedule after an operation, on the operation group: Resolve(0) and,
// after every fourth, Resolve(1); after every fourth Resolve(1) the deep
// group takes over Resolve(2).
template <class Team>
__device__ void conc_schedule(Team &t, Smem &S, OpsCtl &c)
{
    HeapState &hs = S.hs;
    const int q = (int)hs.q;
    if (hs.L[0].slen > 0) {
        {
            PhaseTimer<Team> pt(t, STAT_T_EMPTY);
            empty_level_once(t, S, 0);
        }
        // an S_1 pushed over capacity is emptied on the spot; that pushes
        // into S_2, which the operation group must own first
        if (q > 1 && hs.L[1].slen > hs.L[1].capS && !t.failed()) {
            if (c.deep) own_level2(t, S, c);
            conc_empty_cascade(t, S, c, 1);
        }
    }
    resolve_fill(t, S, 0);
    if (q > 1 && hs.L[0].nres % 4 == 0 && !t.failed()) {
        if (c.deep) {
            // the Resolve(2) released last has finished; Resolve(1) touches
            // levels 1 and 2 only (a cascade past S_2 takes the deeper ones)
            own_level2(t, S, c);
            if (hs.L[1].slen > 0) {
                PhaseTimer<Team> pt(t, STAT_T_DEEP);
                conc_empty_cascade(t, S, c, 1);
            }
            resolve_fill(t, S, 1);
        } else {
            resolve(t, S, 1);
        }
        // Resolve(1) number j has just finished.  The count is read after
        // resolve_fill's closing barrier: its leader thread updates it with no
        // barrier before, so a read ahead of the call could see either value
        // and split the CTA over the release below.
        const u64 j = hs.L[1].nres;
        if (q > 2 && !c.deep) {
            // no deep group: the deeper resolves run here, in order
            for (int i = 2; i < q && !t.failed(); i++) {
                if (hs.L[i - 1].nres % 4 != 0) break;
                resolve(t, S, i);
            }
        } else if (c.deep && j % 4 == 0 && !t.failed()) {
            t.sync();
            deep_release(t, S, c, j / 4);
        }
    }
}

// Before an extract of r: B_0 holds at least r elements, or the fill cascade
// over every level runs (while the deep group is idle).
template <class Team>
__device__ void conc_ensure_top(Team &t, Smem &S, u64 r, OpsCtl &c)
{
    if (S.hs.L[0].blen >= r) return;
    if (c.deep) {
        own_all_levels(t, S, c);
        c.dirty = true;
    }
    ensure_top(t, S, r);
}

// The operation group: every operation of ops[0, nops) in order, each
// followed by its share of the schedule; then the deep group is stopped once
// idle and the whole heap state is written back.
template <class Team>
__device__ void run_ops(Team &t, Smem &S, HeapCounters *cnt, const OpDesc *ops, u32 nops, OpsCtl &c)
{
    HeapState &hs = S.hs;
    const u64 gtid = (u64)t.cta() * NT + threadIdx.x, stride = (u64)t.ncta() * NT;
    for (u32 k = 0; k < nops && !t.failed(); k++) {
        const OpDesc op = ops[k];
        if (op.kind == OP_BULK) {
            // update(e) for every e (min-semantics), staging the words that
            // lower a key's live word for S_0, as a single BulkUpdate does
            u64 fresh_local = 0;
            for (u64 base = (u64)t.cta() * NT; base < op.count; base += stride) {
                const u64 i = base + threadIdx.x;
                bool imp = false;
                u64 P = 0;
                if (i < op.count) {
                    const u32 key = op.keys[i];
                    if (key >= hs.key_space) {
                        raise_err(t.sc.err, ST_INVAL, 11);
                    } else {
                        P = ((u64)op.prios[i] << 32) | key;
                        const u64 old = atomicMin(hs.cur + key, P);
                        imp = old > P;
                        fresh_local += (old == INF);
                    }
                }
                block_emit(imp, P, hs.U[0], hs.d, t.sc.ucount, t.sc.err, S);
            }
            fresh_local = block_sum(fresh_local, S);
            if (threadIdx.x == 0 && fresh_local) atomicAdd(&cnt->inserted, fresh_local);
            t.sync();
            if (t.failed()) break;
            bulk_sort(t, S, ldg_cg(t.sc.ucount));
            if (t.failed()) break;
            conc_schedule(t, S, c);
        } else {
            conc_ensure_top(t, S, op.r, c);
            if (t.failed()) break;
            Level &L0 = hs.L[0];
            const u64 n = L0.blen < op.r ? L0.blen : op.r;
            const u64 *F = L0.B[L0.bsel] + L0.bhead;
            for (u64 j = gtid; j < n; j += stride) {
                const u64 x = ldg_cg(F + j);
                const u32 key = (u32)(x & 0xffffffffu);
                op.kout[j] = key;
                op.pout[j] = (u32)(x >> 32);
                if (hs.reset_on_extract) hs.cur[key] = INF;
            }
            if (gtid == 0) {
                *op.nout = (u32)n;
                cnt->extracted += n;
            }
            __syncthreads();
            LEADER
            {
                L0.bhead += n;
                L0.blen -= n;
            }
            t.sync();
            conc_schedule(t, S, c);
        }
    }
    // wind down: take every deep level back (the deep group is then idle and
    // the state here is current), stop it, and write the whole state back
    if (c.deep) own_all_levels(t, S, c);
    if (t.cta() == 0 && threadIdx.x == 0) *(volatile u32 *)&c.ds->stop = 1;
    t.sync();
    if (t.cta() == 0) state_store(S, c.g_hs);
}

// The deep group: Resolve(2) number j once released, then the deeper
// resolves it triggers; until the operation group stops it.  A wait for the
// next release is bounded (SPIN_NS).
template <class Team>
__device__ void deep_serve(Team &t, Smem &S, HeapState *g_hs, DeepSync *ds)
{
    for (u64 j = 1;; j++) {
        if (threadIdx.x == 0) {
            u64 go = 0, t0 = 0;
            for (u32 spins = 0;; spins++) {
                if (ld_acquire(&ds->ready) >= j) {
                    go = 1;
                    break;
                }
                if (*(volatile u32 *)&ds->stop) break;
                if ((spins & 255) == 0) {
                    if (read_err(t.sc.err) != 0) break;
                    const u64 now = gtimer();
                    if (t0 == 0) {
                        t0 = now;
                    } else if (now - t0 > SPIN_NS) {
                        raise_err(t.sc.err, ST_TIMEOUT, 31);
                        break;
                    }
                }
            }
            S.bc[0] = go;
            S.bc[1] = go ? *(volatile u32 *)&ds->dirty : 0;
        }
        __syncthreads();
        const bool go = S.bc[0] != 0;
        const bool reload_all = S.bc[1] == j;
        __syncthreads();
        if (!go) break;
        // level 2 from the operation group; the deeper ones are this group's
        // own unless the operation group changed them
        levels_load(S, g_hs, 2, reload_all ? 0 : 3);
        resolve(t, S, 2);
        t.sync(); // every CTA's merges are complete
        if (t.cta() == 0) {
            levels_store(S, g_hs, 2, 3);
            __syncthreads();
            if (threadIdx.x == 0) st_release(&ds->done, j);
        }
        for (int i = 3; i < (int)S.hs.q && !t.failed(); i++) {
            if (S.hs.L[i - 1].nres % 4 != 0) break;
            resolve(t, S, i);
        }
        t.sync();
        if (t.cta() == 0) {
            levels_store(S, g_hs, 3);
            __syncthreads();
            if (threadIdx.x == 0) st_release(&ds->idle, j);
        }
        if (t.failed()) break;
    }
}

} // namespace pbhk
