"""Concurrent resolution of non-adjacent levels (Section 2.2.1, Figure 2,
Theorem 3) through pbh_run_ops: a whole operation stream in one launch, the
deep levels resolved by their own CTA group while the operation group keeps
going.  Every extract is compared op by op with the sorted-array oracle, the
level invariants are checked at the end, and the same stream run phase by
phase (no deep group) and operation by operation gives the same results."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


def record(key_space, batch, r, rounds, seed):
    """A closed-loop stream (the generator learns the extracted keys) with the
    oracle's extract results: [(keys, prios, want_keys, want_prios)]."""
    hs = gen.HeapStream(key_space, seed)
    q = oracle.SortedPQ(key_space)
    out = []
    for _ in range(rounds):
        k, p = hs.next_batch(batch)
        q.bulk_update(k, p)
        wk, wp = q.extract_min(r)
        hs.observe_extracted(wk)
        out.append((k, p, wk, wp))
    return out, len(q)


def run_stream(lib, key_space, d, stream, r, deep_ctas):
    h = lib.Heap(key_space, d)
    ops = []
    for k, p, _, _ in stream:
        ops.append(("bulk", k, p))
        ops.append(("extract", r))
    outs = h.run_ops(ops, deep_ctas=deep_ctas)
    got = []
    for ko, po, co in outs:
        n = int(co.item())
        got.append((ko[:n].cpu().numpy().view(np.uint32), po[:n].cpu().numpy().view(np.uint32)))
    return h, got


@pytest.mark.parametrize("deep_ctas", [0, 16, 64])
@pytest.mark.parametrize("key_space,d,batch,r,rounds", [(1 << 12, 16, 16, 5, 400), (1 << 16, 256, 256, 64, 300)])
def test_run_ops_matches_oracle(lib, deep_ctas, key_space, d, batch, r, rounds):
    stream, live = record(key_space, batch, r, rounds, 7 + d)
    h, got = run_stream(lib, key_space, d, stream, r, deep_ctas)
    for i, ((gk, gp), (_, _, wk, wp)) in enumerate(zip(got, stream)):
        assert np.array_equal(gk, wk) and np.array_equal(gp, wp), f"extract {i}"
    viol, _ = h.validate()
    assert viol == 0
    assert h.size() == live
    st = h.stats()
    assert sum(1 for x in st["resolves"] if x) >= 4  # levels 0..3 at least were resolved


def test_run_ops_benchmark_stream_shape(lib):
    # the benchmark heap stream's shape scaled down: key space 2^20, d = 2^12,
    # BulkUpdate(2^12) + extract(2^10), five levels
    stream, live = record(1 << 20, 1 << 12, 1 << 10, 160, 2)
    h, got = run_stream(lib, 1 << 20, 1 << 12, stream, 1 << 10, 32)
    for i, ((gk, gp), (_, _, wk, wp)) in enumerate(zip(got, stream)):
        assert np.array_equal(gk, wk) and np.array_equal(gp, wp), f"extract {i}"
    assert h.validate()[0] == 0
    assert h.size() == live


def test_run_ops_mixed_with_single_operations(lib):
    # one heap driven by single-operation calls and by sequences in turn, and a
    # sequence longer than one launch (4096 operations)
    stream, live = record(1 << 8, 4, 3, 2300, 11)
    h = lib.Heap(1 << 8, 4)
    i = 0
    for chunk in (100, 2100, 100):
        part = stream[i:i + chunk]
        if chunk == 100:
            for k, p, wk, wp in part:
                h.bulk_update(k, p)
                gk, gp = h.extract_min(3)
                assert np.array_equal(gk, wk) and np.array_equal(gp, wp)
        else:
            ops = []
            for k, p, _, _ in part:
                ops += [("bulk", k, p), ("extract", 3)]
            outs = h.run_ops(ops, deep_ctas=16)
            for (ko, po, co), (_, _, wk, wp) in zip(outs, part):
                n = int(co.item())
                assert np.array_equal(ko[:n].cpu().numpy().view(np.uint32), wk)
                assert np.array_equal(po[:n].cpu().numpy().view(np.uint32), wp)
        i += chunk
    assert h.validate()[0] == 0
    assert h.size() == live


def test_run_ops_rejects_bad_operations(lib):
    import ctypes
    h = lib.Heap(1 << 10, 8)
    so = lib.load()
    arr = (lib._Op * 1)()
    arr[0] = lib._Op(7, 0, 0, 0, None, None, None, None, None)
    assert so.pbh_run_ops(h._h, arr, 1, 0) == 1  # PBH_E_INVAL: unknown kind
    arr[0] = lib._Op(lib.OP_EXTRACT, 0, 9, 0, None, None, None, None, None)
    assert so.pbh_run_ops(h._h, arr, 1, 0) == 1  # r > d, null outputs
    assert so.pbh_run_ops(h._h, ctypes.cast(None, ctypes.POINTER(lib._Op)), 0, 0) == 0
