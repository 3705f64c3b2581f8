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
