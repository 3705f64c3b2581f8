// heapop.cuh -- the heap-API operations on a team (one operation and its
// resolves; the debug validator).  The kernels of k_op.cu wrap them; the CPU
// emulation tests call them directly.
#pragma once
#include "core.cuh"

namespace pbhk {

// One heap operation of the pbh API (BulkUpdate, assign, delete or
// extract) followed by Resolve(0) and the Theorem 3 schedule, on a team
// that holds the whole heap.  g_hs is the state in global memory (loaded
// here, stored back at the end); cnt the monotone counters.
template <class Team>
__device__ void heap_op(Team &t, Smem &S, HeapState *g_hs, HeapCounters *cnt, int op, const u32 *keys,
                        const u32 *prios, u32 count, u32 r, u32 *kout, u32 *pout, u32 *nout)
{
    state_load(S, g_hs);
    HeapState &hs = S.hs;
    const u64 gtid = (u64)t.cta() * NT + threadIdx.x, stride = (u64)t.ncta() * NT;
    if (read_err(t.sc.err) != 0) return; // a latched error makes the heap read-only
    if (op == OP_BULK) {
        // update(e) for every e: the live word of a key only ever decreases;
        // a word that lowers it is staged for S_0 (Section 2.2: BulkUpdate
        // inserts into S_0).
        u64 fresh_local = 0;
        for (u64 base = (u64)t.cta() * NT; base < count; base += stride) {
            const u64 i = base + threadIdx.x;
            bool imp = false;
            u64 P = 0;
            if (i < count) {
                const u32 k = keys[i];
                if (k >= hs.key_space) {
                    raise_err(t.sc.err, ST_INVAL, 11);
                } else {
                    P = ((u64)prios[i] << 32) | k;
                    const u64 old = atomicMin(hs.cur + k, P);
                    imp = old > P;
                    fresh_local += (old == INF);
                }
            }
            block_emit(imp, P, hs.U[0], hs.d, t.sc.ucount, t.sc.err, S);
        }
        fresh_local = block_sum(fresh_local, S);
        if (threadIdx.x == 0 && fresh_local) atomicAdd(&cnt->inserted, fresh_local);
        t.sync();
        if (!t.failed()) {
            const u64 nu = ldg_cg(t.sc.ucount);
            LEADER hs.live = ldg_cg(&cnt->inserted) - ldg_cg(&cnt->extracted) - ldg_cg(&cnt->deleted);
            __syncthreads();
            bulk_commit(t, S, nu);
        }
    } else if (op == OP_DELETE) {
        // delete(e) (Section 1.2): the key stops being live.  The paper sends
        // a DEL element down the levels; here the key's entry in cur becomes
        // INF, which makes every stored copy stale at once, and each merge
        // that meets a copy drops it.  B_0 is filtered now, so that extract
        // never returns a deleted key.
        u64 gone = 0;
        for (u64 i = gtid; i < count; i += stride) {
            const u32 k = keys[i];
            if (k >= hs.key_space)
                raise_err(t.sc.err, ST_INVAL, 11);
            else
                gone += atomicExch(hs.cur + k, INF) != INF;
        }
        gone = block_sum(gone, S);
        if (threadIdx.x == 0 && gone) atomicAdd(&cnt->deleted, gone);
        t.sync();
        if (!t.failed()) {
            LEADER hs.live = ldg_cg(&cnt->inserted) - ldg_cg(&cnt->extracted) - ldg_cg(&cnt->deleted);
            __syncthreads();
            if (hs.L[0].blen > 0) empty_level_once(t, S, 0); // S_0 is empty: this drops B_0's stale words
            if (!t.failed()) resolve_schedule(t, S);
        }
    } else if (op == OP_ASSIGN) {
        // update(e) with the replace of Section 1.2's footnote: e replaces
        // its key's element, up or down, and of several elements of one key
        // the latest (here: the last in the batch) wins.  The batch is sorted
        // as (key << 32 | position) words; the last word of each key applies
        // its element to cur and stages it if the live word changed; the
        // replaced copies are stale from then on.
        for (u64 i = gtid; i < count; i += stride) {
            const u32 k = keys[i];
            if (k >= hs.key_space) {
                raise_err(t.sc.err, ST_INVAL, 11);
                hs.U[0][i] = INF; // sorts last, applies nothing
            } else {
                hs.U[0][i] = ((u64)k << 32) | i;
            }
        }
        t.sync();
        u64 *srt = t.failed() ? hs.U[0] : team_sort(t, S, hs.U[0], count, hs.U[1]);
        const int stage = srt == hs.U[0] ? 1 : 0; // the staged words go to the other buffer
        u64 fresh_local = 0;
        if (!t.failed()) {
            for (u64 base = (u64)t.cta() * NT; base < count; base += stride) {
                const u64 j = base + threadIdx.x;
                bool imp = false;
                u64 W = 0;
                if (j < count) {
                    const u64 w = ldg_cg(srt + j);
                    const bool last = j + 1 == count || (ldg_cg(srt + j + 1) >> 32) != (w >> 32);
                    if (w != INF && last) {
                        const u32 k = (u32)(w >> 32), i = (u32)w;
                        W = ((u64)prios[i] << 32) | k;
                        const u64 old = ldg_cg(hs.cur + k); // the only writer of key k in this operation
                        if (old != W) {
                            hs.cur[k] = W;
                            imp = true;
                            fresh_local += old == INF;
                        }
                    }
                }
                block_emit(imp, W, hs.U[stage], hs.d, t.sc.ucount, t.sc.err, S);
            }
        }
        fresh_local = block_sum(fresh_local, S);
        if (threadIdx.x == 0 && fresh_local) atomicAdd(&cnt->inserted, fresh_local);
        t.sync();
        if (!t.failed()) {
            const u64 nu = ldg_cg(t.sc.ucount);
            LEADER hs.live = ldg_cg(&cnt->inserted) - ldg_cg(&cnt->extracted) - ldg_cg(&cnt->deleted);
            __syncthreads();
            bulk_commit(t, S, nu, stage);
        }
    } else {
        ensure_top(t, S, r);
        Level &L0 = hs.L[0];
        const u64 n = L0.blen < r ? L0.blen : r;
        const u64 *F = L0.B[L0.bsel] + L0.bhead;
        for (u64 j = gtid; j < n; j += stride) {
            const u64 x = ldg_cg(F + j);
            const u32 k = (u32)(x & 0xffffffffu);
            kout[j] = k;
            pout[j] = (u32)(x >> 32);
            if (hs.reset_on_extract) hs.cur[k] = INF;
        }
        if (gtid == 0) {
            *nout = (u32)n;
            cnt->extracted += n;
        }
        __syncthreads();
        LEADER
        {
            L0.bhead += n;
            L0.blen -= n;
            hs.live -= n;
        }
        t.sync();
        resolve_schedule(t, S);
    }
    t.sync();
    if (t.cta() == 0) state_store(S, g_hs);
}

// Debug check of the heap invariants by one CTA (all its threads call it).
// Valid copies are counted once per key: a key that pbh_assign sets back to
// a word it held before while a stale copy of that word is still stored
// deeper makes that copy valid again, and the two equal copies coexist until
// a merge meets them (extract stays exact: B_0 never holds both, and
// extracting one invalidates the other).  Pass 1 counts the distinct valid
// keys and marks the keys with more than one valid copy (bitmaps seen and
// dup, zeroed by the caller); pass 2 checks the level order of every key
// stored once.
__device__ inline void heap_validate(Smem &S, const HeapState *g_hs, u32 *viol, u64 *stored, u64 *nvalid, u32 *seen,
                              u32 *dup)
{
    state_load(S, g_hs);
    const HeapState &hs = S.hs;
    u32 bad = 0;
    u64 st = 0, nv = 0;
    for (int pass = 0; pass < 2; pass++) {
        u64 tprev = 0; // max threshold of the shallower levels
        bool have_tprev = false;
        for (u32 i = 0; i < hs.q; i++) {
            const Level &L = hs.L[i];
            if (pass == 0) {
                if (L.blen > L.capB) bad |= 8;
                if (L.slen > L.bufS || L.bhead + L.blen > L.bufB || L.shead + L.slen > L.bufS) bad |= 8;
                if (i > 0 && hs.L[i - 1].T != INF && L.T != INF && L.T < hs.L[i - 1].T && L.blen) bad |= 64;
            }
            for (int which = 0; which < 2; which++) {
                const u64 *R = which == 0 ? L.B[L.bsel] + L.bhead : L.S[L.ssel] + L.shead;
                const u64 len = which == 0 ? L.blen : L.slen;
                if (pass == 0) st += len;
                for (u64 j = threadIdx.x; j < len; j += NT) {
                    const u64 x = R[j];
                    const u64 key = x & hs.keymask;
                    const bool valid = key < hs.key_space && hs.cur[key] == x;
                    const u32 bit = 1u << (key & 31);
                    if (pass == 0) {
                        if (j > 0 && R[j - 1] > x) bad |= 1;
                        if (!valid) {
                            if (i == 0 && which == 0) bad |= 32;
                            continue;
                        }
                        if (atomicOr(seen + (key >> 5), bit) & bit)
                            atomicOr(dup + (key >> 5), bit); // a further copy of a returned word
                        else
                            nv++;
                    } else {
                        if (!valid || (dup[key >> 5] & bit)) continue;
                        if (which == 0 && L.T != INF && x > L.T) bad |= 2;
                        if (have_tprev && x <= tprev) bad |= 4;
                    }
                }
                __syncthreads();
            }
            // every element stored deeper must exceed T_i; an unbounded T_i
            // (INF) leaves no room below it, so any deeper element is a violation
            if (!have_tprev || L.T > tprev) tprev = L.T;
            have_tprev = true;
        }
    }
    atomicOr(viol, bad);
    atomicAdd(stored, st);
    atomicAdd(nvalid, nv);
}


} // namespace pbhk
