"""GPU parity of the parallel bucket heap (pbh_* through the C ABI) against the
sorted-array oracle, op by op.  Extract outputs are unique once ties are
broken by key, so every extract must match exactly."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


def drive(lib, key_space, d, batch, r, rounds, seed, validate=False, capacity=0):
    h = lib.Heap(key_space, d, capacity)
    q = oracle.SortedPQ(key_space)
    hs = gen.HeapStream(key_space, seed)
    for i in range(rounds):
        k, p = hs.next_batch(batch)
        h.bulk_update(k, p)
        q.bulk_update(k, p)
        if validate:
            v, _ = h.validate()
            assert v == 0, (i, "after update", v)
        gk, gp = h.extract_min(r)
        wk, wp = q.extract_min(r)
        assert np.array_equal(gk, wk) and np.array_equal(gp, wp), i
        hs.observe_extracted(wk)
        if validate:
            v, _ = h.validate()
            assert v == 0, (i, "after extract", v)
    assert h.size() == len(q)
    return h, q


@pytest.mark.parametrize("d,batch,r,rounds", [(16, 16, 4, 300), (64, 64, 16, 200), (256, 200, 100, 60),
                                              (1024, 1024, 256, 40)])
def test_stream_small(lib, d, batch, r, rounds):
    drive(lib, 1 << 12, d, batch, r, rounds, seed=d, validate=True)


def test_drain_to_empty(lib):
    h, q = drive(lib, 1 << 10, 32, 32, 8, 100, seed=5)
    while len(q):
        gk, gp = h.extract_min(32)
        wk, wp = q.extract_min(32)
        assert np.array_equal(gk, wk) and np.array_equal(gp, wp)
    gk, _ = h.extract_min(32)
    assert len(gk) == 0 and h.size() == 0


def test_semantics(lib):
    from tests.test_oracle import load_pq_fixture
    ks, ops = load_pq_fixture("pq_hand.txt")
    h = lib.Heap(ks, 8)
    last = None
    for op, arg in ops:
        if op == "update":
            h.bulk_update(np.array([k for k, _ in arg], np.uint32), np.array([p for _, p in arg], np.uint32))
        elif op == "extract":
            last = h.extract_min(arg)
        elif op == "expect":
            assert list(zip(last[0].tolist(), last[1].tolist())) == arg
        elif op == "size":
            assert h.size() == arg


def test_ties_duplicates_and_reinsert(lib):
    h = lib.Heap(64, 16)
    q = oracle.SortedPQ(64)
    batches = [([5, 5, 6, 7], [10, 3, 3, 3]), ([5, 6], [3, 2]), ([8, 9, 10], [0, 0, 0])]
    for k, p in batches:
        k, p = np.array(k, np.uint32), np.array(p, np.uint32)
        h.bulk_update(k, p)
        q.bulk_update(k, p)
    for r in (2, 1, 16):
        a, b = h.extract_min(r), q.extract_min(r)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # re-insert extracted keys with the same priorities they had
    k, p = np.array([8, 6], np.uint32), np.array([0, 2], np.uint32)
    h.bulk_update(k, p)
    q.bulk_update(k, p)
    a, b = h.extract_min(16), q.extract_min(16)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_errors(lib):
    h = lib.Heap(100, 8)
    with pytest.raises(lib.PbhError) as e:
        h.bulk_update(np.zeros(9, np.uint32), np.zeros(9, np.uint32))
    assert e.value.status == 1
    with pytest.raises(lib.PbhError):
        h.extract_min(9)
    h.bulk_update(np.array([100], np.uint32), np.array([1], np.uint32))
    with pytest.raises(lib.PbhError) as e:
        h.sync()
    assert e.value.status == 1


def test_benchmark_stream_shape_short(lib):
    # key space 2^24, d = 2^16 batches of 2^16 pairs, extract 2^14: the
    # first rounds of the full op stream, op by op, with invariant checks
    drive(lib, 1 << 24, 1 << 16, 1 << 16, 1 << 14, 40, seed=2, validate=True)


@pytest.mark.slow
def test_benchmark_stream_full(lib):
    drive(lib, 1 << 24, 1 << 16, 1 << 16, 1 << 14, 1000, seed=2)
