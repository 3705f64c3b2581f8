"""Concurrent resolution of non-adjacent levels (Section 2.2.1, Figure 2,
Theorem 3) on the CPU: run_ops and deep_serve of concurrent.cuh compiled for
the host (tests/emu) and run as one emulated cooperative launch, an operation
group and a deep group of CTAs, over a closed-loop BulkUpdate + extract
stream.  Every extract is compared with the sorted-array oracle, the level
invariants are checked at the end, and the deep levels must have been
resolved (by the deep group) for the test to count."""
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


@pytest.fixture(scope="module")
def ops_harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("emu_ops")
    try:
        exe = host_headers.build("ops_harness", str(d), ())
    except FileNotFoundError:
        pytest.skip("g++ not available")
    except RuntimeError as e:
        pytest.fail(str(e))
    return exe, d


def record(key_space, batch, r, rounds, seed):
    """A closed-loop stream (the generator learns the extracted keys) and the
    oracle's extract results: [(keys, prios, want_keys, want_prios)], live."""
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


def run_ops(harness, key_space, d, stream, r, ctas, n_op):
    exe, tmp = harness
    ip, op = str(tmp / f"ops_{n_op}.bin"), str(tmp / f"out_{n_op}.bin")
    with open(ip, "wb") as f:
        np.array([key_space, d, 2 * len(stream)], dtype=np.uint64).tofile(f)
        for k, p, _, _ in stream:
            np.array([0, len(k), 0], dtype=np.uint64).tofile(f)
            np.asarray(k, np.uint32).tofile(f)
            np.asarray(p, np.uint32).tofile(f)
            np.array([1, 0, r], dtype=np.uint64).tofile(f)
    res = subprocess.run([exe, ip, op, str(ctas), str(n_op)], capture_output=True, text=True, timeout=900, env=host_headers.run_env())
    assert res.returncode == 0, res.stderr[-2000:]
    raw = open(op, "rb").read()
    got, pos = [], 0
    for _ in range(2 * len(stream)):
        n = int(np.frombuffer(raw, np.uint64, 1, pos)[0])
        pos += 8
        k = np.frombuffer(raw, np.uint32, n, pos)
        pos += 4 * n
        p = np.frombuffer(raw, np.uint32, n, pos)
        pos += 4 * n
        got.append((k, p))
    viol, stored, valid, live, status, q = (int(x) for x in np.frombuffer(raw, np.uint64, 6, pos))
    nres = [int(x) for x in np.frombuffer(raw, np.uint64, q, pos + 48)]
    return got[1::2], (viol, valid, live, status), nres


@pytest.mark.parametrize("ctas,n_op", [(2, 1), (3, 2)])
def test_concurrent_resolution_emulated(ops_harness, ctas, n_op):
    # key space 2^12, d = 16: five levels, so Resolve(2) runs on the deep
    # group every 16 operations and Resolve(3) behind it (140 operations:
    # 8 of the first, 2 of the second)
    ks, d, r = 1 << 12, 16, 5
    stream, live = record(ks, 16, r, 70, 23)
    got, (viol, valid, hlive, status), nres = run_ops(ops_harness, ks, d, stream, r, ctas, n_op)
    assert status == 0
    for i, ((gk, gp), (_, _, wk, wp)) in enumerate(zip(got, stream)):
        assert np.array_equal(gk, wk) and np.array_equal(gp, wp), f"extract {i}"
    assert viol == 0 and valid == hlive == live
    assert len(nres) >= 4 and nres[2] > 0 and nres[3] > 0, nres


def test_phase_by_phase_emulated(ops_harness):
    # the operation group alone (no deep group) runs the whole schedule, in
    # order: the same extracts
    ks, d, r = 1 << 12, 16, 5
    stream, live = record(ks, 16, r, 70, 29)
    got, (viol, valid, hlive, status), nres = run_ops(ops_harness, ks, d, stream, r, 2, 2)
    assert status == 0
    for i, ((gk, gp), (_, _, wk, wp)) in enumerate(zip(got, stream)):
        assert np.array_equal(gk, wk) and np.array_equal(gp, wp), f"extract {i}"
    assert viol == 0 and valid == hlive == live
    assert nres[2] > 0
