"""The persistent server's device code on the CPU: the body of k_serve on a
few emulated CTAs, fed by a host thread that fills a request ring as
srv_submit does (the record, then the tail) and reuses a slot only after its
completion flag reports the request before it; then the stop word.  More
requests than slots and than CTAs, so slots are reused while other requests
run.  Every request's distances must equal the oracle's and every request
must have reported its completion.  The same for k_serve_cluster, each
request on one emulated thread-block cluster."""
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
def serve_harness(tmp_path_factory):
    d = tmp_path_factory.mktemp("emu_serve")
    try:
        exe = host_headers.build("serve_harness", str(d), ())
    except FileNotFoundError:
        pytest.skip("g++ not available")
    except RuntimeError as e:
        pytest.fail(str(e))
    return exe, d


def serve(harness, nreq, ctas, slots, cluster, seed):
    exe, tmp = harness
    st = gen.Stream(seed)
    pool = [gen.grid(12, 12, 1, 100, 1), gen.banded(600, 8, 32, 1, 65535, 2),
            gen.random_graph(300, 2400, 1, 1000, 3), gen.grid(1, 1, 1, 1, 4)]
    reqs = []
    for _ in range(nreq):
        g = pool[st.uniform(0, len(pool) - 1)]
        reqs.append((g, st.uniform(0, g.n - 1), 32, 64))
    ip, op = str(tmp / "q.bin"), str(tmp / "out.bin")
    with open(ip, "wb") as f:
        np.array([len(reqs)], dtype=np.uint64).tofile(f)
        for g, s, r, d in reqs:
            np.array([g.n, g.m, s, r, d], dtype=np.uint64).tofile(f)
            g.row_ptr.astype(np.uint64).tofile(f)
            g.col.astype(np.uint32).tofile(f)
            g.w.astype(np.uint32).tofile(f)
    res = subprocess.run([exe, ip, op, str(ctas), str(slots), str(cluster)], capture_output=True, text=True,
                         timeout=900, env=host_headers.run_env())
    assert res.returncode == 0, res.stderr[-2000:]
    raw = open(op, "rb").read()
    pos = 0
    for i, (g, s, _, _) in enumerate(reqs):
        status, flagged = (int(x) for x in np.frombuffer(raw, np.uint64, 2, pos))
        pos += 16
        dist = np.frombuffer(raw, np.uint64, g.n, pos)
        pos += 8 * g.n
        assert status == 0 and flagged == 1, (i, status, flagged)
        assert np.array_equal(dist, oracle.dijkstra(g, s)), i


def test_request_ring_emulated(serve_harness):
    # k_serve: three CTAs, four slots, ten requests
    serve(serve_harness, 10, 3, 4, 1, 4242)


def test_request_ring_clusters_emulated(serve_harness):
    # k_serve_cluster: two clusters of two CTAs, three slots, six requests;
    # the claim is read by the second CTA through distributed shared memory
    serve(serve_harness, 6, 4, 3, 2, 4343)
