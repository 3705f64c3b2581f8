"""Batched mode: many independent queries in one persistent launch
(sssp_batch_run), each checked bit-exactly against the oracle, and each
result identical alone and in the mix."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu


def mixed_queries(k, seed):
    st = gen.Stream(seed)
    graphs, sources = [], []
    for q in range(k):
        if q % 2 == 0:
            side = st.uniform(8, 64)
            g = gen.grid(side, side, 1, 65535, 1000 + q)
        else:
            n = 1 << st.uniform(8, 13)
            g = gen.banded(n, st.uniform(4, 32), 64, 1, 65535, 1000 + q)
        graphs.append(g)
        sources.append(st.uniform(0, g.n - 1))
    return graphs, sources


@pytest.mark.parametrize("r,d", [(0, 0), (8, 512), (1, 64)])
def test_batch_matches_oracle(lib, r, d):
    graphs, sources = mixed_queries(24, 7 + r)
    b = lib.Batch([lib.DeviceGraph(g) for g in graphs], sources, r=r, d=d)
    out = b.run()
    for g, s, got in zip(graphs, sources, out):
        assert np.array_equal(got, oracle.dijkstra(g, s))


def test_batch_mix_invariance(lib):
    graphs, sources = mixed_queries(16, 99)
    dgs = [lib.DeviceGraph(g) for g in graphs]
    mixed = lib.Batch(dgs, sources, r=16, d=1024).run()
    for i, (dg, s) in enumerate(zip(dgs, sources)):
        alone_batch = lib.Batch([dg], [s], r=16, d=1024).run()[0]
        alone_run = lib.sssp(dg, s, r=16, d=1024, cta=1)
        assert np.array_equal(mixed[i], alone_batch)
        assert np.array_equal(mixed[i], alone_run)


def test_batch_more_queries_than_ctas(lib):
    # more queries than resident CTAs: the work queue hands them out in waves
    graphs, sources = [], []
    for q in range(700):
        g = gen.grid(6 + q % 5, 7, 1, 9, q)
        graphs.append(g)
        sources.append(q % g.n)
    out = lib.Batch([lib.DeviceGraph(g) for g in graphs], sources, r=4, d=64).run()
    for g, s, got in zip(graphs[::37], sources[::37], out[::37]):
        assert np.array_equal(got, oracle.dijkstra(g, s))


def test_batch_benchmark_sizes_match_oracle(lib):
    # The largest members of the 512-query benchmark batch (a 512x512 grid,
    # the biggest banded graphs) plus a banded graph of 2^18 vertices at
    # degree 64, each on its one-CTA team with the autotuned r and d, and a
    # seeded sample of the rest, every distance against the oracle.
    import bench
    from paper_1908_09378_gb300 import autotune
    specs = bench.batch_specs()
    grids = sorted((i for i, s in enumerate(specs) if s[0] == "grid"), key=lambda i: -specs[i][1])
    bands = sorted((i for i, s in enumerate(specs) if s[0] == "banded"), key=lambda i: -specs[i][1] * specs[i][2])
    st = gen.Stream(77)
    pick = sorted(set(grids[:2] + bands[:3] + [st.uniform(0, len(specs) - 1) for _ in range(8)]))
    graphs = [bench.make_spec_graph(specs[i]) for i in pick]
    sources = [specs[i][4] for i in pick]
    graphs.append(gen.banded(1 << 18, 64, 256, 1, 65535, 4242))
    sources.append(12345)
    assert max(g.n for g in graphs) >= 512 * 512
    dgs = [lib.DeviceGraph(g) for g in graphs]
    rs, ds, cs = autotune.batch_params(dgs)
    assert max(cs) >= 2  # the largest queries run on clusters
    out = lib.Batch(dgs, sources, r=rs, d=ds, cta=cs).run()
    for g, s, got in zip(graphs, sources, out):
        assert np.array_equal(got, oracle.dijkstra(g, s)), g.name


@pytest.mark.parametrize("k", [2, 4, 8])
def test_batch_cluster_teams_match_oracle(lib, k):
    # queries on k-CTA clusters beside one-CTA queries, in one batch (two
    # launches on two streams); each result exact and equal to the query alone
    graphs, sources = mixed_queries(18, 50 + k)
    graphs += [gen.banded(1 << 14, 48, 256, 1, 65535, 60 + k), gen.grid(120, 120, 1, 65535, 61 + k)]
    sources += [5, 77]
    ctas = [k if i % 3 == 0 or i >= 18 else 1 for i in range(len(graphs))]
    dgs = [lib.DeviceGraph(g) for g in graphs]
    out = lib.Batch(dgs, sources, r=64, d=4096, cta=ctas).run()
    for g, s, got in zip(graphs, sources, out):
        assert np.array_equal(got, oracle.dijkstra(g, s))
    for i in (0, 18, 19):
        assert np.array_equal(out[i], lib.sssp(dgs[i], sources[i], r=64, d=4096, cta=k))
