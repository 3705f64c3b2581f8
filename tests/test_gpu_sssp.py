"""GPU parity of parDijkstra (sssp_run through the C ABI) against the oracle.

Distances are exact integers: the bar is bit-exact equality everywhere."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


def run(lib, g, s, **kw):
    dg = lib.DeviceGraph(g)
    return lib.sssp(dg, s, with_stats=True, **kw)


@pytest.mark.parametrize("r,cta", [(1, 0), (7, 0), (64, 0), (1024, 0), (64, 1), (1024, 1)])
def test_grid64_config(lib, r, cta):
    g = gen.grid(64, 64, 1, 100, 0)
    want = oracle.dijkstra(g, 0)
    got, st = run(lib, g, 0, r=r, d=4096, cta=cta)
    assert np.array_equal(got, want)
    assert st["status"] == 0
    if r == 1:  # paper-faithful: one vertex per round, every reached vertex once
        assert st["rounds"] == g.n and st["extracted"] == g.n


@pytest.mark.parametrize("cta", [0, 1, 4])
@pytest.mark.parametrize("side", [2, 4, 8, 16])
def test_small_grids_one_per_round(lib, side, cta):
    # Dijkstra proper (r = 1) on tiny grids, for every team: one vertex per
    # round, every vertex once, B_0 slices thinner than one word per CTA
    g = gen.grid(side, side, 1, 100, side)
    want = oracle.dijkstra(g, 0)
    got, st = run(lib, g, 0, r=1, d=64, cta=cta)
    assert np.array_equal(got, want)
    assert st["status"] == 0 and st["rounds"] == g.n


@pytest.mark.parametrize("cta", [0, 1, 4])
def test_settle_grid64_r1(lib, cta):
    # r = 1 with the settle criterion: the same distances in fewer rounds
    g = gen.grid(64, 64, 1, 100, 0)
    want = oracle.dijkstra(g, 0)
    got, st = run(lib, g, 0, r=1, d=4096, cta=cta, flags=lib.SSSP_SETTLE)
    assert np.array_equal(got, want)
    assert st["settled"] > 0 and st["rounds"] < g.n
    assert st["rounds"] + st["settled"] == st["extracted"]


def test_settle_paper_dag(lib):
    # on the paper's DAG vertex v + 1 gets its distance v + 1 only from v's
    # chain arc, so nothing beyond the minimum is ever final: one per round
    g = gen.dag(2000, 60000)
    want = oracle.dijkstra(g, 0)
    got, st = run(lib, g, 0, r=1, d=4 * g.max_degree, flags=lib.SSSP_SETTLE)
    assert np.array_equal(got, want)
    assert st["rounds"] == g.n and st["settled"] == 0


@pytest.mark.parametrize("seed", range(4))
def test_settle_random_with_zero_weights(lib, seed):
    st_ = gen.Stream(5150 + seed)
    n = st_.uniform(2, 2500)
    g = gen.random_graph(n, st_.uniform(0, 6 * n), 0, [0, 1, 5, 1000][seed], seed)
    s = st_.uniform(0, n - 1)
    want = oracle.dijkstra(g, s)
    got, st = run(lib, g, s, r=[1, 2, 8, 1][seed], d=max(g.max_degree, 1) * 16, cta=seed % 2,
                  flags=lib.SSSP_SETTLE)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("seed", range(12))
def test_random_graphs(lib, seed):
    st_ = gen.Stream(4242 + seed)
    n = st_.uniform(1, 3000)
    m = st_.uniform(0, 8 * n)
    g = gen.random_graph(n, m, 0 if seed % 2 else 1, 1000, seed)
    s = st_.uniform(0, n - 1)
    want = oracle.dijkstra(g, s)
    r = [1, 3, 32, 256][seed % 4]
    d = max(g.max_degree, 1) * [1, 2, 5, 64][seed % 4]
    got, st = run(lib, g, s, r=r, d=d, cta=seed % 3 == 0)
    assert np.array_equal(got, want)
    assert not oracle.check_sssp(g, s, got).any()


@pytest.mark.parametrize("d", [64, 256, 4096])
def test_many_levels_banded(lib, d):
    # small d => many levels, cascades and on-demand fills are exercised
    g = gen.banded(1 << 14, 16, 64, 1, 65535, 5)
    want = oracle.dijkstra(g, 0)
    got, st = run(lib, g, 0, r=max(1, d // 16), d=d)
    assert np.array_equal(got, want)
    assert st["levels"] >= 2


@pytest.mark.parametrize("cta", [2, 4])
@pytest.mark.parametrize("d", [64, 128])
def test_many_levels_cluster(lib, d, cta):
    # few CTAs per team: each CTA merges several tiles in turn (the multi-tile
    # path of the team merge) while levels 1..3 fill and empty
    g = gen.random_graph(2000, 16000, 1, 1000, 9) if d == 128 else gen.banded(1 << 12, 16, 64, 1, 65535, 5)
    s = 3 if d == 128 else 0
    want = oracle.dijkstra(g, s)
    got, st = run(lib, g, s, r=max(1, d // 16), d=d, cta=cta)
    assert np.array_equal(got, want)
    assert st["levels"] >= 3


def test_banded_medium(lib):
    g = gen.banded(1 << 16, 64, 512, 1, 65535, 1)
    want = oracle.dijkstra(g, 0)
    got, st = run(lib, g, 0)
    assert np.array_equal(got, want)
    assert st["relaxations"] >= oracle.reached_edges(g, want)


@pytest.mark.parametrize("d,cta", [(1 << 21, 0), (1 << 16, 0), (1 << 16, 8), (4096, 0)])
def test_query_counters(lib, d, cta):
    # the counters kept in registers and added once per query agree with
    # their definitions, on the single-step rounds (nothing below level 0:
    # d = 2^21, 2^16) and with deeper levels (d = 4096): Resolve(0) runs once
    # per round plus once for the source, every merged word is kept or
    # dropped as stale, every scanned arc is counted once
    g = gen.banded(1 << 16, 32, 256, 1, 65535, 4)
    want = oracle.dijkstra(g, 0)
    got, st = run(lib, g, 0, r=min(128, d // 32), d=d, cta=cta)
    assert np.array_equal(got, want)
    assert st["resolves"][0] == st["rounds"] + 1, st
    assert 0 < st["stale_dropped"] < st["merged"], st
    assert st["relaxations"] >= oracle.reached_edges(g, want), st
    assert st["improvements"] >= int((want != np.uint64(2**64 - 1)).sum()) - 1, st
    a = run(lib, g, 0, r=min(128, d // 32), d=d, cta=cta)[1]
    assert a["relaxations"] == st["relaxations"] and a["rounds"] == st["rounds"]


def test_banded_full_size(lib):
    # the n = 2^20, degree-64, window +-512 graph in the launch configuration
    # the benchmark times (default options, whole-GPU cooperative launch)
    g = gen.banded(1 << 20, 64, 512, 1, 65535, 1)
    want = oracle.dijkstra(g, 0)
    got, st = run(lib, g, 0)
    assert np.array_equal(got, want)
    assert st["status"] == 0


def test_paper_dag(lib):
    n, m = 3000, 400000
    g = gen.dag(n, m, 11)
    got, st = run(lib, g, 0, r=1, d=g.max_degree)
    assert np.array_equal(got, np.arange(n, dtype=np.uint64))
    got, st = run(lib, g, 0, r=64, d=64 * g.max_degree)
    assert np.array_equal(got, np.arange(n, dtype=np.uint64))


def test_hand_fixture(lib):
    from tests.test_oracle import load_sssp_fixture
    g, s, want, _ = load_sssp_fixture("sssp_hand6.txt")
    for r in (1, 2, 6):
        got, _ = run(lib, g, s, r=r, d=8)
        assert np.array_equal(got, want)


def test_edge_cases(lib):
    # single vertex, no arcs
    g = gen.random_graph(1, 0, 1, 1, 0)
    got, _ = run(lib, g, 0)
    assert got.tolist() == [0]
    # source without out-arcs: everything else unreachable
    g = gen.grid(4, 4, 1, 9, 0)
    rp = g.row_ptr.copy()
    g2 = gen.Graph(g.n, np.concatenate([[0], np.full(g.n, 0)]).astype(np.uint64), g.col[:0], g.w[:0])
    got, _ = run(lib, g2, 3)
    assert got[3] == 0 and (np.delete(got, 3) == oracle.INF).all()
    # zero weights everywhere
    g = gen.grid(16, 16, 0, 0, 0)
    got, _ = run(lib, g, 5, r=16, d=64)
    assert (got == 0).all()


def test_errors(lib):
    g = gen.grid(8, 8, 1, 9, 0)
    dg = lib.DeviceGraph(g)
    with pytest.raises(lib.PbhError) as e:
        lib.sssp(dg, 64)
    assert e.value.status == 1  # source >= n
    with pytest.raises(lib.PbhError) as e:
        lib.sssp(dg, 0, r=4, d=2)  # d below the largest out-degree
    assert e.value.status == 1
    # distances that do not fit the packed word: 2^20 vertices leave 44 bits
    n = 1 << 20
    rp = np.arange(n + 1, dtype=np.uint64)
    rp[-1] = n - 1
    col = np.arange(1, n, dtype=np.uint32)
    w = np.full(n - 1, 0xFFFFFFFF, dtype=np.uint32)
    big = gen.Graph(n, rp, col, w)
    with pytest.raises(lib.PbhError) as e:
        lib.sssp(lib.DeviceGraph(big), 0, r=1024, d=1024)
    assert e.value.status == 4


def test_host_entry_point(lib):
    g = gen.banded(1 << 15, 32, 256, 1, 65535, 9)
    want = oracle.dijkstra(g, 7)
    got, _ = lib.sssp_host(g, 7)
    assert np.array_equal(got[: g.n], want)


def test_deterministic_stats(lib):
    # The words that survive into S_0 each round are the new minima, which do
    # not depend on the order concurrent atomicMin operations land in, so the
    # rounds, extractions and scanned arcs repeat exactly.  The number of
    # successful atomicMin calls (improvements) legitimately varies.
    g = gen.banded(1 << 15, 32, 256, 1, 65535, 9)
    a = run(lib, g, 0)[1]
    b = run(lib, g, 0)[1]
    for k in ("rounds", "extracted", "relaxations"):
        assert a[k] == b[k], k


@pytest.mark.parametrize("name", ["grid64", "banded14"])
def test_library_chosen_team(lib, name):
    # opts = NULL: the library picks the team by size (a 16-CTA cluster for
    # the 64x64 grid, the whole GPU for 2^20 arcs); distances exact either way
    g = gen.grid(64, 64, 1, 100, 0) if name == "grid64" else gen.banded(1 << 14, 64, 512, 1, 65535, 1)
    dg = lib.DeviceGraph(g)
    got, st = lib.sssp(dg, 0, with_stats=True, auto=True)
    assert np.array_equal(got, oracle.dijkstra(g, 0))


@pytest.mark.parametrize("cta", [17, 76])
def test_grid_of_given_size(lib, cta):
    # a cooperative grid of exactly `cta` CTAs (fewer than one per SM)
    g = gen.banded(1 << 13, 32, 128, 1, 65535, 6)
    dg = lib.DeviceGraph(g)
    got = lib.sssp(dg, 3, r=256, d=1 << 14, cta=cta)
    assert np.array_equal(got, oracle.dijkstra(g, 3))



def test_phase_times_heap_only(lib):
    # heap operations record their device time per phase; the query teams
    # compile the timers out (their t_*_ns stay 0) and give the same distances
    g = gen.banded(1 << 12, 16, 64, 1, 1000, 5)
    dg = lib.DeviceGraph(g)
    want = oracle.dijkstra(g, 0)
    for cta in (0, 4, 1):
        got, st = lib.sssp(dg, 0, r=64, cta=cta, with_stats=True)
        assert np.array_equal(got, want)
        assert st["t_relax_ns"] == 0 and st["t_empty0_ns"] == 0, (cta, st)
    h = lib.Heap(1 << 12, 64)
    h.bulk_update(np.arange(64, dtype=np.uint32), np.arange(64, dtype=np.uint32)[::-1].copy())
    h.extract_min(8)
    assert h.stats()["t_sort_ns"] + h.stats()["t_empty0_ns"] > 0
