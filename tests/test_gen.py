"""The seeded input generators: determinism and the shapes of each recipe."""
import numpy as np
import pytest

import gen


def test_determinism():
    a = gen.banded(5000, 16, 64, 1, 65535, 3)
    b = gen.banded(5000, 16, 64, 1, 65535, 3)
    c = gen.banded(5000, 16, 64, 1, 65535, 4)
    assert np.array_equal(a.col, b.col) and np.array_equal(a.w, b.w)
    assert not np.array_equal(a.w, c.w)


def test_grid_shape():
    g = gen.grid(64, 64, 1, 100, 0)
    assert g.n == 4096 and g.m == 16128
    assert g.w.min() >= 1 and g.w.max() <= 100
    for v in [0, 63, 64 * 63, 4095, 1000]:
        r, c = divmod(v, 64)
        nb = sorted(x for x, ok in [(v - 64, r > 0), (v - 1, c > 0), (v + 1, c < 63), (v + 64, r < 63)] if ok)
        assert g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist() == nb


@pytest.mark.parametrize("n,deg,win", [(3000, 64, 512), (70, 16, 256), (1000, 7, 3)])
def test_banded_shape(n, deg, win):
    g = gen.banded(n, deg, win, 1, 65535, 1)
    for i in range(n):
        t = g.col[g.row_ptr[i]:g.row_ptr[i + 1]].astype(np.int64)
        cand = min(n - 1, i + win) - max(0, i - win)
        assert len(t) == min(deg, cand)
        assert (np.diff(t) > 0).all()
        assert (np.abs(t - i) <= win).all() and (t != i).all()
        assert t.min(initial=0) >= 0 and t.max(initial=0) < n
    assert g.w.min() >= 1 and g.w.max() <= 65535


def test_banded_full_size_edges():
    assert gen._load().gen_banded_edges(1 << 20, 64, 512) == 1 << 26


def test_dag_shape():
    n, m = 200, 5000
    g = gen.dag(n, m, 0)
    assert g.m == m
    for u in range(n - 1):
        t = g.col[g.row_ptr[u]:g.row_ptr[u + 1]].astype(np.int64)
        w = g.w[g.row_ptr[u]:g.row_ptr[u + 1]].astype(np.int64)
        assert t[0] == u + 1 and w[0] == 1
        assert (np.diff(t) > 0).all() and (t > u).all()
        assert (w[1:] == 2 * (t[1:] - u)).all()
    deg = np.diff(g.row_ptr.astype(np.int64))
    # extra arcs spread evenly over the sources that are not saturated
    cap = (n - 1) - np.arange(n - 1)
    unsat = deg[:-1] < cap
    assert deg[:-1][unsat].max() - deg[:-1][unsat].min() <= 1


def test_heap_stream_batches():
    hs = gen.HeapStream(1 << 10, 2)
    k, p = hs.next_batch(256)
    assert len(k) == 256 and len(np.unique(k)) == 256
    rec = dict(zip(k.tolist(), p.tolist()))
    k2, p2 = hs.next_batch(256)
    assert len(np.unique(k2)) == len(k2)
    dec = [(a, b) for a, b in zip(k2.tolist(), p2.tolist()) if a in rec]
    assert len(dec) == 128
    assert all(b < rec[a] for a, b in dec)
