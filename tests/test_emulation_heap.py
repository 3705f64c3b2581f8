"""The heap-API device code on the CPU: heap_op and heap_validate of
heapop.cuh compiled for the host (tests/emu) and run on a few emulated CTAs
joined by the grid-team barrier, one operation after another, against the
sorted-array oracle: every extract's pairs, the validator's invariants and
the live count after every operation."""
import os
import subprocess
import sys

import numpy as np
import pytest

import gen
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "emu"))
import host_headers  # noqa: E402

KINDS = {"update": 0, "extract": 1, "delete": 2, "assign": 3}


def _build(tmp_path_factory, defines=()):
    d = tmp_path_factory.mktemp("emu_heap")
    try:
        exe = host_headers.build("heap_harness", str(d), defines)
    except FileNotFoundError:
        pytest.skip("g++ not available")
    except RuntimeError as e:
        pytest.fail(str(e))
    return exe, d


@pytest.fixture(scope="module")
def heap_harness(tmp_path_factory):
    return _build(tmp_path_factory)


@pytest.fixture(scope="module")
def heap_harness_tiles(tmp_path_factory):
    # merge tiles loaded by bulk copies (alignment checked on the host)
    return _build(tmp_path_factory, ["-DPBH_BULK_TILES"])


def run_stream(heap_harness, key_space, d, ops, ctas=3):
    """ops: (kind, keys, prios, r) tuples.  Returns, per operation, the
    extracted (keys, prios) and (violations, stored, valid keys, live)."""
    exe, tmp = heap_harness
    ip, op = str(tmp / "ops.bin"), str(tmp / "out.bin")
    with open(ip, "wb") as f:
        np.array([key_space, d, len(ops)], dtype=np.uint64).tofile(f)
        for kind, keys, prios, r in ops:
            np.array([KINDS[kind], len(keys), r], dtype=np.uint64).tofile(f)
            np.asarray(keys, np.uint32).tofile(f)
            np.asarray(prios, np.uint32).tofile(f)
    res = subprocess.run([exe, ip, op, str(ctas)], capture_output=True, text=True, timeout=900, env=host_headers.run_env())
    assert res.returncode == 0, res.stderr[-2000:]
    raw = open(op, "rb").read()
    out, pos = [], 0
    for _ in ops:
        n = int(np.frombuffer(raw, np.uint64, 1, pos)[0])
        pos += 8
        k = np.frombuffer(raw, np.uint32, n, pos)
        pos += 4 * n
        p = np.frombuffer(raw, np.uint32, n, pos)
        pos += 4 * n
        rec = np.frombuffer(raw, np.uint64, 4, pos)
        pos += 32
        out.append(((k, p), tuple(int(x) for x in rec)))
    return out


def general_stream(key_space, d, nops, seed):
    """The mixed stream of the GPU general-operations test: BulkUpdate,
    assign, delete and extract over a small key space (every batch collides
    with live keys), with narrow priority ranges every third operation."""
    st = gen.Stream(31337 + seed)
    ops = []
    for i in range(nops):
        kind = st.uniform(0, 3)
        cnt = st.uniform(0, d)
        keys = gen.uniform_u32(cnt, 0, key_space - 1, st.next())
        hi = 15 if i % 3 == 0 else (1 << 32) - 1
        prios = gen.uniform_u32(cnt, 0, hi, st.next())
        if kind == 3:
            ops.append(("extract", np.zeros(0, np.uint32), np.zeros(0, np.uint32), st.uniform(0, d)))
        else:
            ops.append((("update", "assign", "delete")[kind], keys, prios if kind != 2 else np.zeros(cnt, np.uint32),
                        0))
    return ops


def check_against_oracle(out, ops, key_space):
    q = oracle.SortedPQ(key_space)
    for i, ((kind, keys, prios, r), (got, (viol, stored, valid, live))) in enumerate(zip(ops, out)):
        if kind == "update":
            q.bulk_update(keys, prios)
        elif kind == "assign":
            q.assign(keys, prios)
        elif kind == "delete":
            q.delete(keys)
        else:
            want = q.extract_min(r)
            assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1]), (i, "extract")
        assert viol == 0 and valid == live, (i, kind, viol, valid, live)
        assert live == len(q), (i, kind, live, len(q))


@pytest.mark.parametrize("key_space,d,nops,seed", [(64, 16, 120, 1), (512, 64, 70, 2)])
def test_general_stream_emulated(heap_harness, key_space, d, nops, seed):
    ops = general_stream(key_space, d, nops, seed)
    check_against_oracle(run_stream(heap_harness, key_space, d, ops), ops, key_space)


def test_assign_back_to_an_earlier_word_emulated(heap_harness):
    # key 0 at priority 1000 is pushed several levels down by smaller
    # elements, moves to priority 5, then back to 1000: the stale copy of its
    # first word, still stored deep, is valid again beside the new one; the
    # key is counted once and extracted once
    ks, d = 256, 4
    none = np.zeros(0, np.uint32)
    ops = [("assign", np.array([0], np.uint32), np.array([1000], np.uint32), 0)]
    for base in range(1, 200, 4):
        keys = np.arange(base, base + 4, dtype=np.uint32)
        ops.append(("update", keys, (keys % 50).astype(np.uint32), 0))
    ops.append(("assign", np.array([0], np.uint32), np.array([5], np.uint32), 0))
    ops.append(("assign", np.array([0], np.uint32), np.array([1000], np.uint32), 0))
    ops += [("extract", none, none, 3) for _ in range(67)]
    check_against_oracle(run_stream(heap_harness, ks, d, ops), ops, ks)


def test_large_batches(heap_harness):
    # BulkUpdate and assign batches above one tile (2048 words) on 8 CTAs:
    # the team sort's merge passes, then Empty(S_0) of a batch several tiles
    # long
    d, ks = 4096, 1 << 16
    st = gen.Stream(77)
    none = np.zeros(0, np.uint32)
    ops = []
    for i in range(6):
        cnt = 2500 + 250 * i
        keys = gen.uniform_u32(cnt, 0, ks - 1, st.next())
        prios = gen.uniform_u32(cnt, 0, (1 << 20) if i % 2 else 255, st.next())
        ops.append(("update", keys, prios, 0))
        ops.append(("extract", none, none, 1500))
    ops += [("assign", gen.uniform_u32(3000, 0, ks - 1, st.next()), gen.uniform_u32(3000, 0, 1000, st.next()), 0)]
    ops += [("extract", none, none, d) for _ in range(6)]
    check_against_oracle(run_stream(heap_harness, ks, d, ops, ctas=8), ops, ks)



def test_general_stream_bulk_tiles(heap_harness_tiles):
    ops = general_stream(64, 16, 120, 1)
    check_against_oracle(run_stream(heap_harness_tiles, 64, 16, ops), ops, 64)
