"""The batched kernel's device code on the CPU: the body of k_sssp_batch (a
work queue over the longest-first run order, each claimed query run by
run_query on its own heap with the one-CTA team, CtaTeam) compiled for the
host (tests/emu) on a few emulated CTAs.  Every query's distances must equal
the oracle's.  This is the only CPU coverage of the one-CTA team's paths
(block sort, inline merges, no team barriers), which the batched and served
kernels run; and the body of k_sssp_batch_cluster, each query on one
emulated thread-block cluster (ClusterTeam) whose first CTA claims it."""
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
def batch_harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("emu_batch")
    try:
        exe = host_headers.build("batch_harness", str(d), ())
    except FileNotFoundError:
        pytest.skip("g++ not available")
    except RuntimeError as e:
        pytest.fail(str(e))
    return exe, d


def run_batch(harness, queries, ctas, cluster=1):
    """queries: (graph, source, r, d).  Returns per query (status, rounds,
    levels, distances)."""
    exe, tmp = harness
    ip, op = str(tmp / "q.bin"), str(tmp / "out.bin")
    with open(ip, "wb") as f:
        np.array([len(queries)], dtype=np.uint64).tofile(f)
        for g, s, r, d in queries:
            np.array([g.n, g.m, s, r, d], dtype=np.uint64).tofile(f)
            g.row_ptr.astype(np.uint64).tofile(f)
            g.col.astype(np.uint32).tofile(f)
            g.w.astype(np.uint32).tofile(f)
    res = subprocess.run([exe, ip, op, str(ctas), str(cluster)], capture_output=True, text=True, timeout=900, env=host_headers.run_env())
    assert res.returncode == 0, res.stderr[-2000:]
    raw = open(op, "rb").read()
    out, pos = [], 0
    for g, _, _, _ in queries:
        st, rounds, levels = (int(x) for x in np.frombuffer(raw, np.uint64, 3, pos))
        pos += 24
        out.append((st, rounds, levels, np.frombuffer(raw, np.uint64, g.n, pos)))
        pos += 8 * g.n
    return out


def test_batch_work_queue_emulated(batch_harness):
    # more queries than CTAs, of mixed sizes and shapes: r = 1 (one vertex a
    # round), wide frontiers, batches of more than one tile, and small d
    # (three levels: Empty and Fill below level 0 on one CTA)
    queries = [
        (gen.grid(8, 8, 1, 100, 1), 0, 1, 64),
        (gen.grid(32, 32, 1, 100, 2), 517, 64, 64),
        (gen.banded(2000, 16, 64, 1, 1000, 3), 11, 512, 2048),
        (gen.random_graph(800, 6400, 1, 1000, 5), 3, 128, 256),
        (gen.random_graph(400, 1600, 0, 3, 6), 7, 64, 64),  # zero weights, many ties
        (gen.dag(100, 1000, 7), 0, 32, 64),
        (gen.grid(1, 1, 1, 1, 8), 0, 4, 16),                # a single vertex
    ]
    got = run_batch(batch_harness, queries, 3)
    for i, ((g, s, _, _), (st, rounds, levels, dist)) in enumerate(zip(queries, got)):
        assert st == 0, (i, st)
        assert np.array_equal(dist, oracle.dijkstra(g, s)), i
    assert got[0][1] >= queries[0][0].n          # r = 1: a round per vertex
    assert max(lv for _, _, lv, _ in got) >= 3    # small d: the deeper levels ran


def test_batch_clusters_emulated(batch_harness):
    # two clusters of two CTAs take five queries: the claim goes through the
    # first CTA's shared memory, every query runs on its cluster's team
    queries = [
        (gen.grid(16, 16, 1, 100, 11), 3, 16, 64),
        (gen.banded(2000, 16, 64, 1, 1000, 12), 5, 256, 4096),
        (gen.random_graph(600, 4800, 1, 1000, 13), 0, 32, 64),
        (gen.grid(1, 1, 1, 1, 14), 0, 4, 16),
        (gen.banded(1024, 8, 32, 1, 65535, 15), 100, 64, 128),
    ]
    got = run_batch(batch_harness, queries, 4, cluster=2)
    for i, ((g, s, _, _), (st, _, _, dist)) in enumerate(zip(queries, got)):
        assert st == 0, (i, st)
        assert np.array_equal(dist, oracle.dijkstra(g, s)), i
