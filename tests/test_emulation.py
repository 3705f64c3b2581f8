"""The device code's control flow on the CPU: run_query of core.cuh compiled
for the host (tests/emu: every CUDA thread a std::thread, shared memory per
emulated CTA, the grid-team barrier on real atomics) with a few CTAs, so that
each CTA merges several tiles and the heap's deeper levels fill and empty.
Distances must equal the oracle's.  A race between the threads of a CTA (a
value read after another thread overwrote it) shows up here as a latched
error, a stall or a wrong distance, without a GPU."""
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


def _build_harness(tmp_path_factory, defines=()):
    d = tmp_path_factory.mktemp("emu")
    try:
        exe = host_headers.build("harness", str(d), defines)
    except FileNotFoundError:
        pytest.skip("g++ not available")
    except RuntimeError as e:
        pytest.fail(str(e))
    return exe, d


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    return _build_harness(tmp_path_factory)


@pytest.fixture(scope="module")
def harness_bulk(tmp_path_factory):
    # relax staging arc rows into shared memory with bulk copies (on the host
    # a copy completes at once)
    return _build_harness(tmp_path_factory, ["-DPBH_BULK_RELAX"])


def emulate(harness, g, s, r, d, ctas=3, settle=0, cluster=False, stall=False, limit_ms=0, expect_rc=0):
    exe, tmp = harness
    gp, op = str(tmp / "g.bin"), str(tmp / "d.bin")
    with open(gp, "wb") as f:
        np.array([g.n, g.m, s, r, d], dtype=np.uint64).tofile(f)
        g.row_ptr.astype(np.uint64).tofile(f)
        g.col.astype(np.uint32).tofile(f)
        g.w.astype(np.uint32).tofile(f)
    res = subprocess.run([exe, gp, op, str(ctas), str(settle), "1" if cluster else "0", "1" if stall else "0",
                          str(limit_ms)], capture_output=True, text=True, timeout=600, env=host_headers.run_env())
    assert res.returncode == expect_rc, res.stderr[-2000:]
    return np.fromfile(op, dtype=np.uint64), res.stderr


def test_grid_team_small_d(harness):
    # d = 64: several levels; r = 16: fused sort + Empty of the batch
    g = gen.grid(32, 32, 1, 100, 1)
    got, _ = emulate(harness, g, 5, 16, 64, 3)
    assert np.array_equal(got, oracle.dijkstra(g, 5))


def test_grid_team_deeper_levels(harness):
    # the live set outgrows B_0 within a few rounds: pushes into S_1, Empty(1),
    # Fill(0) from level 1, on three CTAs.  A merge that let one thread
    # overwrite the tile start before the others had read it latched a bad
    # key here within 11 rounds.
    g = gen.random_graph(1000, 8000, 1, 1000, 9)
    got, err = emulate(harness, g, 3, 8, 128, 3)
    assert np.array_equal(got, oracle.dijkstra(g, 3))
    assert "levels 3" in err


def test_grid_team_settle(harness):
    g = gen.grid(8, 8, 1, 100, 5)
    got, err = emulate(harness, g, 0, 1, 64, 3, settle=1)
    assert np.array_equal(got, oracle.dijkstra(g, 0))
    assert " settled 0" not in err


def test_bulk_staged_relax(harness_bulk):
    # degree-16 rows start on 16-byte boundaries: every row is staged; the
    # random multigraph's rows mostly are not: plain loads beside staged rows
    g = gen.banded(4096, 16, 64, 1, 1000, 3)
    got, _ = emulate(harness_bulk, g, 7, 64, 2048, 3)
    assert np.array_equal(got, oracle.dijkstra(g, 7))
    h = gen.random_graph(800, 6400, 1, 1000, 4)
    got, _ = emulate(harness_bulk, h, 1, 16, 256, 3)
    assert np.array_equal(got, oracle.dijkstra(h, 1))


def test_grid_team_wide_batches(harness):
    # wide frontiers stage more than one tile of improved vertices per round
    # on 8 CTAs: the general BulkUpdate path (team sort with the words
    # gathered from the distance array, then Empty(S_0))
    g = gen.random_graph(6000, 96000, 1, 1000, 21)
    got, _ = emulate(harness, g, 4, 256, 8192, 8)
    assert np.array_equal(got, oracle.dijkstra(g, 4))


@pytest.fixture(scope="module")
def harness_tiles(tmp_path_factory):
    # merge tiles loaded by bulk copies (on the host a copy completes at once
    # and aborts if its addresses or size are not 16-byte multiples)
    return _build_harness(tmp_path_factory, ["-DPBH_BULK_TILES"])


def test_bulk_tile_loads(harness_tiles):
    # many-level heap merges, and the team sort's merge passes of wide
    # batches, with every tile's runs at all word parities
    g = gen.random_graph(1000, 8000, 1, 1000, 9)
    got, err = emulate(harness_tiles, g, 3, 8, 128, 3)
    assert np.array_equal(got, oracle.dijkstra(g, 3))
    assert "levels 3" in err
    h = gen.random_graph(6000, 96000, 1, 1000, 21)
    got, _ = emulate(harness_tiles, h, 4, 256, 8192, 8)
    assert np.array_equal(got, oracle.dijkstra(h, 4))


def test_cluster_team(harness):
    # one thread-block cluster of 4 CTAs (ClusterTeam, the hardware cluster
    # barrier emulated as one barrier over all the cluster's threads): several
    # levels on the grid, and a frontier wide enough for the team sort's
    # merge passes on the random multigraph
    g = gen.grid(24, 24, 1, 100, 3)
    got, err = emulate(harness, g, 17, 16, 64, 4, cluster=True)
    assert np.array_equal(got, oracle.dijkstra(g, 17))
    assert "levels 3" in err
    h = gen.random_graph(3000, 40000, 1, 1000, 22)
    got, _ = emulate(harness, h, 9, 256, 4096, 4, cluster=True)
    assert np.array_equal(got, oracle.dijkstra(h, 9))


def test_bounded_waits_expire(harness):
    # the failure path of the grid barrier's bounded wait, without a GPU: one
    # arrival short (CTA 0 withholds it; every wait is bounded by 200 ms).
    # Each CTA's thread 0 latches PBH_E_TIMEOUT at the barrier site between
    # the barrier's two CTA-wide syncs, so every CTA winds down on the same
    # branch: the process exits with the latched status (5), no stall.  The
    # query time limit is not run here: its check raises the error from one
    # thread in the middle of a barrier interval in which the other threads
    # may still read the error state, so on the way out a CTA can split over
    # its barriers, which a CTA whose exited threads do not count as arrived
    # (this emulation) waits on.
    g = gen.grid(16, 16, 1, 100, 7)
    for _ in range(3):
        _, err = emulate(harness, g, 0, 16, 64, 3, stall=True, expect_rc=5)
        assert "status 5 site 1 " in err, err
