"""Served mode: one persistent launch, queries published as they arrive,
admitted by device-memory footprint.  Every result must equal the oracle
and the same query run alone (mix invariance)."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


def pool(k, seed):
    st = gen.Stream(seed)
    gs = []
    for q in range(k):
        if q % 2:
            gs.append(gen.banded(1 << st.uniform(9, 13), 32, 256, 1, 65535, 500 + q))
        else:
            side = st.uniform(16, 80)
            gs.append(gen.grid(side, side, 1, 65535, 500 + q))
    return gs


def requests_for(graphs, n, rate, seed):
    from paper_1908_09378_gb300.serve import poisson_arrivals
    st = gen.Stream(seed + 1)
    arr = poisson_arrivals(n, rate, seed)
    reqs = []
    for a in arr:
        gi = st.uniform(0, len(graphs) - 1)
        reqs.append((a, gi, st.uniform(0, graphs[gi].n - 1)))
    return reqs


def test_served_results_match_oracle_and_alone(lib):
    from paper_1908_09378_gb300 import serve
    graphs = pool(12, 3)
    dgs = [lib.DeviceGraph(g) for g in graphs]
    reqs = requests_for(graphs, 150, 3000.0, 7)
    got = {}
    sv = serve.Server(budget_bytes=2 << 30, slots=256)
    try:
        stats = serve.run_stream(sv, dgs, reqs, collect=lambda i, d: got.__setitem__(i, d.cpu().numpy().view(np.uint64)),
                                 check_status=True)
    finally:
        sv.stop()
    assert stats["served"] == 150
    for i, (_, gi, src) in enumerate(reqs):
        want = oracle.dijkstra(graphs[gi], src)
        assert np.array_equal(got[i], want), i
    # mix invariance: the same queries alone, one sssp_run each
    for i in range(0, 150, 15):
        _, gi, src = reqs[i]
        r, d = serve.params_for(dgs[gi])
        alone = lib.sssp(dgs[gi], src, r=r, d=d, cta=1)
        assert np.array_equal(got[i], alone)


def test_admission_under_small_budget(lib):
    # a budget that holds only a few queries at a time: everything still
    # completes, and the pool never holds more than the budget
    from paper_1908_09378_gb300 import serve
    graphs = pool(6, 11)
    dgs = [lib.DeviceGraph(g) for g in graphs]
    sv0 = serve.Server(budget_bytes=1 << 20, slots=16)
    fp = max(sum(sv0.footprint(g, *serve.params_for(g))) for g in dgs)
    sv0.stop()
    budget = 3 * fp
    reqs = requests_for(graphs, 60, 1e9, 13)  # all at once
    sv = serve.Server(budget_bytes=budget, slots=64)
    got = {}
    try:
        stats = serve.run_stream(sv, dgs, reqs, collect=lambda i, d: got.__setitem__(i, d.cpu().numpy().view(np.uint64)))
    finally:
        sv.stop()
    assert stats["served"] == 60
    assert stats["peak_pool_bytes"] <= budget
    for i in range(0, 60, 7):
        _, gi, src = reqs[i]
        assert np.array_equal(got[i], oracle.dijkstra(graphs[gi], src))


def test_served_benchmark_sizes_match_oracle(lib):
    # The served pool at its extremes: a 1024x1024 grid and a banded graph of
    # 2^20 vertices (degree 32, window +-256) beside small graphs, each query
    # on one CTA with the autotuned parameters; every result against the oracle.
    from paper_1908_09378_gb300 import serve
    graphs = [gen.grid(1024, 1024, 1, 65535, 2001), gen.banded(1 << 20, 32, 256, 1, 65535, 2033),
              gen.grid(40, 40, 1, 65535, 2002), gen.banded(1 << 12, 32, 256, 1, 65535, 2034)]
    dgs = [lib.DeviceGraph(g) for g in graphs]
    st = gen.Stream(5)
    reqs = [(0.0, gi, st.uniform(0, graphs[gi].n - 1)) for gi in (0, 1, 2, 3, 1, 0, 3, 2)]
    for large_team in (0, 4):
        # without and with the cluster launch for graphs of >= 2^20 arcs
        got = {}
        sv = serve.Server(budget_bytes=8 << 30, slots=64, large_team=large_team, large_ctas=16, large_arcs=1 << 20)
        try:
            stats = serve.run_stream(sv, dgs, reqs,
                                     collect=lambda i, d: got.__setitem__(i, d.cpu().numpy().view(np.uint64)),
                                     check_status=True)
        finally:
            sv.stop()
        assert stats["served"] == len(reqs)
        for i, (_, gi, src) in enumerate(reqs):
            assert np.array_equal(got[i], oracle.dijkstra(graphs[gi], src)), (large_team, i, graphs[gi].name)


def test_cluster_server_alone_vs_mix(lib):
    # the cluster launch serves large queries in the mix; each result equals
    # the same query run alone on a cluster of the same size
    from paper_1908_09378_gb300 import serve
    graphs = pool(10, 21)
    graphs.append(gen.banded(1 << 16, 32, 256, 1, 65535, 2041))
    dgs = [lib.DeviceGraph(g) for g in graphs]
    reqs = requests_for(graphs, 120, 2000.0, 23)
    got = {}
    sv = serve.Server(budget_bytes=4 << 30, slots=128, large_team=2, large_ctas=8, large_arcs=1 << 14)
    try:
        serve.run_stream(sv, dgs, reqs, collect=lambda i, d: got.__setitem__(i, d.cpu().numpy().view(np.uint64)),
                         check_status=True)
    finally:
        sv.stop()
    for i, (_, gi, src) in enumerate(reqs):
        if i % 6 == 0:
            assert np.array_equal(got[i], oracle.dijkstra(graphs[gi], src))
        if dgs[gi].m >= (1 << 14) and i % 4 == 0:
            r, d = serve.params_for(dgs[gi], 2)
            assert np.array_equal(got[i], lib.sssp(dgs[gi], src, r=r, d=d, cta=2))
