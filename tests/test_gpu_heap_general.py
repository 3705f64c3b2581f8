"""GPU parity of the general heap operations against the sorted-array oracle,
op by op: update with the timestamped replace of Section 1.2's footnote
(pbh_assign: the last pair of a key wins, up or down) and delete (pbh_delete),
interleaved with the decrease-only BulkUpdate and extract."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


def same(a, b):
    return np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_general_semantics_fixture(lib):
    from tests.test_oracle import load_pq_fixture
    ks, ops = load_pq_fixture("pq_general.txt")
    h = lib.Heap(ks, 8)
    last = None
    for op, arg in ops:
        if op == "update":
            h.bulk_update(np.array([k for k, _ in arg], np.uint32), np.array([p for _, p in arg], np.uint32))
        elif op == "assign":
            h.assign(np.array([k for k, _ in arg], np.uint32), np.array([p for _, p in arg], np.uint32))
        elif op == "delete":
            h.delete(np.array(arg, np.uint32))
        elif op == "extract":
            last = h.extract_min(arg)
        elif op == "expect":
            assert list(zip(last[0].tolist(), last[1].tolist())) == arg
        elif op == "size":
            assert h.size() == arg


@pytest.mark.parametrize("key_space,d,ops,seed", [(64, 16, 300, 1), (512, 64, 250, 2), (4096, 256, 120, 3),
                                                  (1 << 14, 1024, 60, 4)])
def test_general_stream(lib, key_space, d, ops, seed):
    # small key spaces make every batch collide with live keys: increases,
    # decreases, repeats within a batch, deletes of live and absent keys
    h = lib.Heap(key_space, d)
    q = oracle.SortedPQ(key_space)
    st = gen.Stream(31337 + seed)
    for i in range(ops):
        kind = st.uniform(0, 3)
        cnt = st.uniform(0, d)
        keys = gen.uniform_u32(cnt, 0, key_space - 1, st.next())
        hi = 15 if i % 3 == 0 else (1 << 32) - 1  # narrow ranges force ties
        prios = gen.uniform_u32(cnt, 0, hi, st.next())
        if kind == 0:
            h.bulk_update(keys, prios)
            q.bulk_update(keys, prios)
        elif kind == 1:
            h.assign(keys, prios)
            q.assign(keys, prios)
        elif kind == 2:
            h.delete(keys)
            q.delete(keys)
        else:
            r = st.uniform(0, d)
            assert same(h.extract_min(r), q.extract_min(r)), (i, "extract")
        v, _ = h.validate()
        assert v == 0, (i, kind, v)
        assert h.size() == len(q), (i, kind)
    while len(q):
        assert same(h.extract_min(d), q.extract_min(d))
    assert h.size() == 0 and len(h.extract_min(d)[0]) == 0


def test_delete_front_then_extract(lib):
    # deleting the smallest keys must take them out of B_0 before the next extract
    h = lib.Heap(1 << 10, 64)
    q = oracle.SortedPQ(1 << 10)
    k = np.arange(0, 600, dtype=np.uint32)
    p = (k * 7 + 3).astype(np.uint32)
    for a in range(0, 600, 64):
        h.bulk_update(k[a:a + 64], p[a:a + 64])
        q.bulk_update(k[a:a + 64], p[a:a + 64])
    dead = np.arange(0, 40, dtype=np.uint32)
    h.delete(dead)
    q.delete(dead)
    got = h.extract_min(16)
    assert same(got, q.extract_min(16))
    assert not set(got[0].tolist()) & set(dead.tolist())


def test_assign_raise_moves_key_deeper(lib):
    # raising the current minimum far above everything: it must come out last
    h = lib.Heap(256, 16)
    q = oracle.SortedPQ(256)
    k = np.arange(200, dtype=np.uint32)
    for a in range(0, 200, 16):
        h.bulk_update(k[a:a + 16], k[a:a + 16] + 10)
        q.bulk_update(k[a:a + 16], k[a:a + 16] + 10)
    up = (np.array([0, 1, 2], np.uint32), np.array([1 << 30, 5, 1 << 31], np.uint32))
    h.assign(*up)
    q.assign(*up)
    out = []
    while len(q):
        a, b = h.extract_min(16), q.extract_min(16)
        assert same(a, b)
        out += a[0].tolist()
    assert out[0] == 1 and out[-2:] == [0, 2]


def test_general_errors(lib):
    h = lib.Heap(16, 8)
    with pytest.raises(lib.PbhError):  # count > d
        h.assign(np.arange(9, dtype=np.uint32), np.zeros(9, np.uint32))
    with pytest.raises(lib.PbhError):
        h.delete(np.arange(9, dtype=np.uint32))
    h.assign(np.array([3, 4], np.uint32), np.array([1, 2], np.uint32))  # still usable
    assert h.size() == 2
    h3 = lib.Heap(16, 8)
    h3.assign(np.array([3, 99], np.uint32), np.array([1, 1], np.uint32))  # key >= key_space
    with pytest.raises(lib.PbhError) as e:
        h3.sync()
    assert e.value.status == 1


def test_assign_back_to_an_earlier_word(lib):
    # key 0 gets priority 1000, is pushed below several levels by smaller
    # elements, moves to priority 5, then back to 1000: the stale copy of its
    # first word, still stored deep, is valid again beside the new one.  The
    # heap must still validate (the key counted once), extract the key once,
    # and agree with the oracle throughout.
    ks, d = 256, 4
    h = lib.Heap(ks, d)
    q = oracle.SortedPQ(ks)

    def both(fn, *a):
        getattr(h, fn)(*a)
        getattr(q, fn)(*a)

    both("assign", np.array([0], np.uint32), np.array([1000], np.uint32))
    for base in range(1, 200, 4):
        keys = np.arange(base, base + 4, dtype=np.uint32)
        both("bulk_update", keys, (keys % 50).astype(np.uint32))
        assert h.validate()[0] == 0
    both("assign", np.array([0], np.uint32), np.array([5], np.uint32))
    both("assign", np.array([0], np.uint32), np.array([1000], np.uint32))
    v, _ = h.validate()
    assert v == 0
    assert h.size() == len(q)
    out = []
    while len(q):
        gk, gp = h.extract_min(3)
        wk, wp = q.extract_min(3)
        assert np.array_equal(gk, wk) and np.array_equal(gp, wp)
        out += list(gk)
        assert h.validate()[0] == 0
    assert out.count(0) == 1
    assert h.size() == 0
