"""Continuous-batching SSSP serving over the srv_* C ABI.

One persistent launch serves the queries one CTA each (srv_create); with a
large-query team, a second persistent launch beside it runs the largest
queries one thread-block cluster each (srv_create_team).  This module is the
host-side request loop:

* admission by device-memory footprint: each query needs its heap workspace
  (srv_query_workspace_bytes) plus its distance array; both come from one
  device pool of `budget_bytes` managed by a first-fit allocator, and a
  query is admitted only when its footprint fits (the resident graphs are
  counted once, outside the pool);
* requests are published to the device ring in arrival order as memory and
  ring slots free up, so requests that arrive while others run start as
  soon as a CTA is free and overlap with them on the device;
* completion is detected from the per-slot completion words in mapped host
  memory; latency = completion seen by the host - arrival time.
"""
from __future__ import annotations

import bisect
import ctypes
import time
from collections import deque
from ctypes import POINTER, byref, c_uint32, c_uint64, c_void_p

import numpy as np

import paper_1908_09378_gb300 as pbh

ALIGN = 256


def _up(x: int) -> int:
    return (x + ALIGN - 1) // ALIGN * ALIGN


class FirstFit:
    """First-fit allocator over [0, size) with coalescing free list."""

    def __init__(self, size: int):
        self.size = size
        self.starts = [0]
        self.lens = [size]
        self.used = 0

    def alloc(self, n: int):
        n = _up(n)
        for i, (st, ln) in enumerate(zip(self.starts, self.lens)):
            if ln >= n:
                if ln == n:
                    del self.starts[i]
                    del self.lens[i]
                else:
                    self.starts[i] = st + n
                    self.lens[i] = ln - n
                self.used += n
                return st
        return None

    def free(self, off: int, n: int):
        n = _up(n)
        self.used -= n
        i = bisect.bisect_left(self.starts, off)
        self.starts.insert(i, off)
        self.lens.insert(i, n)
        # coalesce with the right, then the left neighbour
        if i + 1 < len(self.starts) and self.starts[i] + self.lens[i] == self.starts[i + 1]:
            self.lens[i] += self.lens[i + 1]
            del self.starts[i + 1]
            del self.lens[i + 1]
        if i > 0 and self.starts[i - 1] + self.lens[i - 1] == self.starts[i]:
            self.lens[i - 1] += self.lens[i]
            del self.starts[i]
            del self.lens[i]


class _Launch:
    """One persistent server launch (srv_create_team): its ring and completion arrays."""

    def __init__(self, torch, lib, slots, ctas, team, stream):
        self.lib, self.team = lib, team
        self.ws = torch.empty(lib.srv_workspace_bytes(), dtype=torch.uint8, device="cuda")
        self._h = c_void_p()
        pbh._check(lib.srv_create_team(byref(self._h), slots, ctas, team, c_void_p(self.ws.data_ptr()),
                                       self.ws.numel(), c_void_p(stream.cuda_stream)), "srv_create_team")
        d, tb, te = POINTER(c_uint64)(), POINTER(c_uint64)(), POINTER(c_uint64)()
        ns = c_uint32()
        pbh._check(lib.srv_completion_arrays(self._h, byref(d), byref(tb), byref(te), byref(ns)),
                   "srv_completion_arrays")
        self.slots = ns.value
        self.done = np.ctypeslib.as_array(d, shape=(self.slots,))
        self.t_begin = np.ctypeslib.as_array(tb, shape=(self.slots,))
        self.t_end = np.ctypeslib.as_array(te, shape=(self.slots,))

    def stop(self) -> int:
        st = 0
        if self._h.value:
            st = self.lib.srv_stop(self._h)
            self.lib.srv_destroy(self._h)
            self._h = c_void_p()
        return st


class Server:
    """Running persistent servers plus their shared device memory pool.

    Every query runs on one CTA of the main launch, except, with
    large_team >= 2, queries of at least large_arcs arcs: those run on
    thread-block clusters of large_team CTAs in a second launch of large_ctas
    CTAs, beside the first (its CTAs take the remaining SMs, two per SM)."""

    def __init__(self, budget_bytes: int = 40_000_000_000, slots: int = 8192, ctas: int = 0, large_team: int = 0,
                 large_ctas: int = 0, large_arcs: int = 1 << 22):
        torch = pbh._torch()
        lib = pbh.load()
        self.torch, self.lib = torch, lib
        self.pool = torch.empty(budget_bytes, dtype=torch.uint8, device="cuda")
        self.base = self.pool.data_ptr()
        self.alloc = FirstFit(budget_bytes)
        self.budget = budget_bytes
        self.large_team = large_team if large_team >= 2 and large_ctas >= large_team else 0
        self.large_arcs = large_arcs
        self.streams = []
        self.launches = []
        if self.large_team:
            # the cluster launch first: every cluster must be resident
            self.streams.append(torch.cuda.Stream())
            self.launches.append(_Launch(torch, lib, slots, large_ctas, self.large_team, self.streams[-1]))
            if not ctas:
                sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
                ctas = max(1, sms - large_ctas) * 2
        self.streams.append(torch.cuda.Stream())
        self.launches.append(_Launch(torch, lib, slots, ctas, 1, self.streams[-1]))
        self.small = self.launches[-1]
        self.peak_used = 0

    @property
    def _h(self):
        return self.small._h

    @property
    def slots(self):
        return self.small.slots

    def launch_for(self, dg) -> int:
        """Index of the launch that runs queries on this graph."""
        return 0 if self.large_team and dg.m >= self.large_arcs else len(self.launches) - 1

    def footprint(self, dg, r=0, d=0):
        team = self.launches[self.launch_for(dg)].team
        q = pbh._Query(dg.csr(), dg.w.data_ptr(), 0, 8, int(r), int(d), team if team > 1 else 0)
        ws = self.lib.srv_query_workspace_bytes(byref(q))
        return _up(ws), _up(8 * max(dg.n, 1))

    def try_submit(self, dg, source, r=0, d=0):
        """Admit and publish one query if its footprint fits; returns
        ((launch, ticket), off, total_bytes, ws_bytes) or None."""
        li = self.launch_for(dg)
        la = self.launches[li]
        ws_b, dist_b = self.footprint(dg, r, d)
        total = ws_b + dist_b
        off = self.alloc.alloc(total)
        if off is None:
            return None
        dist_ptr = self.base + off + ws_b
        q = pbh._Query(dg.csr(), dg.w.data_ptr(), int(source), dist_ptr, int(r), int(d),
                       la.team if la.team > 1 else 0)
        ticket = c_uint64()
        st = self.lib.srv_submit(la._h, byref(q), c_void_p(self.base + off), ws_b, byref(ticket))
        if st != 0:
            self.alloc.free(off, total)
            if st == 3:  # ring slot busy
                return None
            raise pbh.PbhError(st, "srv_submit", self.lib.pbh_last_error().decode(errors="replace"))
        self.peak_used = max(self.peak_used, self.alloc.used)
        return (li, ticket.value), off, total, ws_b

    def finished(self, keys):
        """The (launch, ticket) keys among `keys` whose query has finished,
        with each one's device run time in ns."""
        out = []
        for li, la in enumerate(self.launches):
            tk = np.fromiter((t for l, t in keys if l == li), dtype=np.uint64)
            if not len(tk):
                continue
            slot = (tk % np.uint64(la.slots)).astype(np.int64)
            fin = la.done[slot] == tk + np.uint64(1)
            for t, sl in zip(tk[fin].tolist(), slot[fin].tolist()):
                out.append(((li, t), float(la.t_end[sl] - la.t_begin[sl])))
        return out

    def heartbeat(self):
        """Tell every launch's waiting CTAs that the host is alive."""
        for la in self.launches:
            if la._h.value:
                self.lib.srv_heartbeat(la._h)

    def dist_of(self, off, ws_b, n):
        """Device distances of a finished query (uint64 bits in an int64 view)."""
        start = off + ws_b
        return self.pool[start:start + 8 * n].view(self.torch.int64)

    def stop(self):
        # every launch is told to stop before any is waited for: a CTA of one
        # launch may be scheduled only when a CTA of the other leaves
        for la in self.launches:
            if la._h.value:
                self.lib.srv_request_stop(la._h)
        st = 0
        for la in self.launches:
            st = la.stop() or st
        if st != 0:
            raise pbh.PbhError(st, "srv_stop", self.lib.pbh_last_error().decode(errors="replace"))

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


def params_for(dg, team: int = 1):
    """(r, d) of a served query on its team: the batch rule's for one CTA,
    the single-query tuner's best on that cluster size for a cluster."""
    from paper_1908_09378_gb300 import autotune
    return autotune.team_params(dg.n, dg.max_degree, team)


def run_stream(server: Server, graphs, requests, collect=None, check_status=False, timeout_s=600.0):
    """Serve `requests` = list of (arrival_s, graph_index, source) in arrival
    order.  `collect(i, dist_tensor)` is called for each finished request if
    given.  Returns a dict with throughput and latency percentiles."""
    n_req = len(requests)
    arrival = np.array([a for a, _, _ in requests], dtype=np.float64)
    params = [params_for(g, server.launches[server.launch_for(g)].team) for g in graphs]
    pending = deque()
    inflight = {}            # ticket -> (req index, off, total, ws_b)
    lat = np.zeros(n_req)
    dev_ns = np.zeros(n_req)
    done_cnt = 0
    nxt = 0
    t0 = time.perf_counter()
    beat = 0.0
    while done_cnt < n_req:
        now = time.perf_counter() - t0
        if now - beat > 0.05:
            server.heartbeat()
            beat = now
        if now > timeout_s:
            raise TimeoutError(f"served {done_cnt}/{n_req} in {timeout_s}s")
        while nxt < n_req and arrival[nxt] <= now:
            pending.append(nxt)
            nxt += 1
        # completions
        if inflight:
            fin = server.finished(list(inflight.keys()))
            if fin:
                tnow = time.perf_counter() - t0
                for t, ns in fin:
                    i, off, total, ws_b = inflight.pop(t)
                    lat[i] = tnow - arrival[i]
                    dev_ns[i] = ns
                    g = graphs[requests[i][1]]
                    if collect is not None:
                        collect(i, server.dist_of(off, ws_b, g.n))
                    if check_status:
                        st = pbh._Stats()
                        code = server.lib.sssp_stats(c_void_p(server.base + off), byref(st),
                                                     pbh._stream(server.torch))
                        if code != 0:
                            raise pbh.PbhError(code, f"served query {i}")
                    server.alloc.free(off, total)
                    done_cnt += 1
        # admissions, in arrival order
        while pending:
            i = pending[0]
            _, gi, src = requests[i]
            r, d = params[gi]
            res = server.try_submit(graphs[gi], src, r, d)
            if res is None:
                break
            ticket, off, total, ws_b = res
            inflight[ticket] = (i, off, total, ws_b)
            pending.popleft()
        if not pending and nxt < n_req and not inflight:
            time.sleep(max(0.0, min(arrival[nxt] - (time.perf_counter() - t0), 0.001)))
    wall = time.perf_counter() - t0
    return {
        "served": n_req, "wall_s": wall, "qps": n_req / wall,
        "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
        "mean_ms": 1e3 * float(lat.mean()), "device_p50_ms": float(np.percentile(dev_ns, 50)) / 1e6,
        "peak_pool_bytes": int(server.peak_used),
    }


def poisson_arrivals(n, rate, seed):
    """n arrival times of a Poisson process with `rate` per second (seeded)."""
    import gen
    st = gen.Stream(seed)
    t, out = 0.0, []
    for _ in range(n):
        u = st.random()
        t += -np.log(1.0 - u) / rate if rate > 0 else 0.0
        out.append(t)
    return out
