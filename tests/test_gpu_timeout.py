"""The bounded device waits, made to run out on purpose, without faulting the
GPU: each test sets a short limit on a wait that cannot finish in time (a
query longer than its time limit, a grid barrier one arrival short, a server
with no request), expects PBH_E_TIMEOUT from the host call that reads the
latched status, and then runs a normal query on the same GPU, which must
match the oracle: the context stays usable."""
import ctypes
import time

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

TIMEOUT = 5  # PBH_E_TIMEOUT


def _check_next_query(lib):
    g = gen.grid(40, 40, 1, 100, 21)
    got = lib.sssp(lib.DeviceGraph(g), 7)
    assert np.array_equal(got, oracle.dijkstra(g, 7))


def test_query_time_limit_expires(lib):
    # r = 1 on a 2^14-vertex banded graph takes 2^14 rounds, far more than 1 ms
    g = gen.banded(1 << 14, 16, 64, 1, 1000, 5)
    dg = lib.DeviceGraph(g)
    for cta in (0, 1, 4):
        with pytest.raises(lib.PbhError) as e:
            lib.sssp(dg, 0, r=1, cta=cta, limit_ms=1)
        assert e.value.status == TIMEOUT, str(e.value)
        assert "site 10" in str(e.value)
    _check_next_query(lib)
    # the same query without the limit finishes and is exact
    assert np.array_equal(lib.sssp(dg, 0, r=1, cta=0), oracle.dijkstra(g, 0))


def test_grid_barrier_wait_expires(lib):
    # the first CTA withholds one barrier arrival: every CTA's 10 ms wait runs out
    g = gen.grid(64, 64, 1, 100, 0)
    dg = lib.DeviceGraph(g)
    t0 = time.perf_counter()
    with pytest.raises(lib.PbhError) as e:
        lib.sssp(dg, 0, cta=0, flags=lib.SSSP_DEBUG_STALL, wait_us=10000)
    assert e.value.status == TIMEOUT, str(e.value)
    assert "site 1)" in str(e.value)  # the grid barrier
    assert time.perf_counter() - t0 < 5.0
    _check_next_query(lib)
    # the stall flag is ignored by the teams without a software barrier
    for cta in (1, 2):
        got = lib.sssp(dg, 0, cta=cta, flags=lib.SSSP_DEBUG_STALL, wait_us=10000)
        assert np.array_equal(got, oracle.dijkstra(g, 0))


def test_server_idle_wait_expires(lib):
    from paper_1908_09378_gb300 import serve
    sv = serve.Server(budget_bytes=64 << 20, slots=16, ctas=4)
    so = lib.load()
    # no request is ever published: every CTA's wait passes the 20 ms bound,
    # the CTAs leave and the server latches the idle timeout
    la = sv.small
    assert so.srv_idle_limit(la._h, 20_000_000) == 0
    time.sleep(0.3)
    st = so.srv_stop(la._h)
    so.srv_destroy(la._h)
    la._h = ctypes.c_void_p()
    assert st == TIMEOUT, so.pbh_last_error()
    _check_next_query(lib)
