#!/usr/bin/env python3
"""Benchmark of parDijkstra driven by the GB300 parallel bucket heap.

Default workload: single-source shortest paths on the banded high-diameter
graph (n = 2^20 vertices, 64 distinct out-arcs per vertex drawn uniformly
from [i-512, i+512], m = 2^26 arcs, uint32 weights uniform in [1, 65535],
seed 1, source 0).  One step = one complete sssp_run (all rounds of
extract-min / relax / BulkUpdate, on the device) with the graph resident in
HBM.  Metric: GTEPS = reached arcs / time.

Other workloads (--workload): grid64 (64x64 grid), dag (the paper's DAG),
heap (bucket-heap op stream: key space 2^24, 2^16-pair BulkUpdates each
followed by an extract of 2^14), heap_general (the same shape with general
updates and deletes), batch (512 mixed queries in one persistent launch),
serve (a Poisson request stream through the persistent server).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
same workload instead (the one place besides the cpu_baseline leg where this
script runs oracle/ code).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------ distributed

class Dist:
    """One process per GPU (torchrun env); only timing reductions cross ranks."""

    def __init__(self, n_gpus: int, backend: str = "nccl"):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        self.n_gpus = n_gpus
        self.backend = backend

    def init(self, torch):
        if self.backend == "nccl":
            torch.cuda.set_device(self.local)
        if self.world > 1:
            import torch.distributed as td
            if self.backend == "nccl":
                td.init_process_group("nccl", device_id=torch.device("cuda", self.local))
            else:
                td.init_process_group(self.backend)
            self.pg = td

    def _dev(self):
        return "cuda" if self.backend == "nccl" else "cpu"

    def barrier(self, torch):
        if self.pg:
            self.pg.barrier()
        if self.backend == "nccl":
            torch.cuda.synchronize()

    def max(self, torch, x: float) -> float:
        if not self.pg:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=self._dev())
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, torch, x: float) -> float:
        if not self.pg:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=self._dev())
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def shard(weights, rank: int, world: int):
    """Indices of the items this rank runs: largest first, each to the rank
    with the least assigned weight so far (greedy LPT).  Deterministic, so
    every rank computes the same partition without communicating."""
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    load = [0] * world
    owner = [0] * len(weights)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += weights[i]
    return [i for i in range(len(weights)) if owner[i] == rank]


# ------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        busy = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(busy), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash() -> str:
    """Hash of the CUDA sources; a committed ncu traffic figure is used only
    while the kernels it was taken on are unchanged."""
    import hashlib
    h = hashlib.sha256()
    for name in ("core.cuh", "pbh.cu", "plan.h"):
        with open(os.path.join(ROOT, "paper_1908_09378_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def committed_traffic(profile_name: str):
    """(bytes per launch, source hash) from a profiles/ summary, or None."""
    p = os.path.join(ROOT, "profiles", profile_name)
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line and line.strip().startswith(("traffic_bytes_per_launch", "kernel_source_hash")):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_hash") != kernel_source_hash() or "traffic_bytes_per_launch" not in vals:
        return None
    return int(vals["traffic_bytes_per_launch"])


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------ workloads

LOGN = 20  # banded workload size (the benchmark line is quoted at 2^20; smaller only for profiling)


def banded_graph():
    return gen.banded(1 << LOGN, 64, 512, 1, 65535, 1)


def banded_cfg():
    return {"workload": f"banded n=2^{LOGN}, 64 distinct out-arcs in [i-512,i+512], m=2^{LOGN + 6}, "
                        "w~U[1,65535] (seed 1), source 0", "n": 1 << LOGN, "m": 1 << (LOGN + 6)}


def algorithmic_bytes(n: int, m: int, reached: int) -> int:
    """Bytes the method must move once: row_ptr (8(n+1)), the arc arrays
    (8m: col + w), the distance write (8n) and one heap word written and read
    per reached vertex (16 per vertex)."""
    return 8 * (n + 1) + 8 * m + 8 * n + 16 * reached


def bench_sssp(args, dist: Dist, torch, pbh):
    if args.workload == "banded":
        g, cfg = banded_graph(), banded_cfg()
    elif args.workload == "dag":
        g = gen.dag(30000, args.m, 0)
        cfg = {"workload": f"the paper's random DAG (Section 4.2): n=30000, m={g.m}, chain of weight 1 plus "
                           "forward arcs of weight 2(v-u), seed 0, source 0", "n": g.n, "m": g.m}
    else:
        g = gen.grid(64, 64, 1, 100, 0)
        cfg = {"workload": "64x64 directed 4-neighbour grid, m=16128, w~U[1,100] (seed 0), source 0",
               "n": g.n, "m": g.m}
    dg = pbh.DeviceGraph(g)
    r, d = args.r, args.d
    if args.workload == "dag" and not r:
        r = 1                                   # the paper's parDijkstra: one vertex per round
    if args.workload == "dag" and not d:
        d = max(1, r) * dg.max_degree           # d = maximum degree (Section 4.1)
    flags = pbh.SSSP_SETTLE if args.settle else 0
    ws = pbh.SsspWorkspace(dg.n, r, d, args.cta, flags=flags)
    distv = torch.empty(dg.n, dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    # warm-up
    for _ in range(args.warmup):
        pbh.sssp_async(dg, 0, dist=distv, ws=ws)
    st = pbh.sssp_stats(ws)
    reached = int((distv != -1).sum().item())
    deg = np.diff(g.row_ptr.astype(np.int64))
    dist_host = distv.cpu().numpy().view(np.uint64)
    m_reached = int(deg[dist_host != np.uint64(0xFFFFFFFFFFFFFFFF)].sum())
    # timed: one event pair per step on the launching stream, L2 flushed between steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(dist.local)
    dist.barrier(torch)
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i)
        starts[i].record(stream)
        pbh.sssp_async(dg, 0, dist=distv, ws=ws)
        ends[i].record(stream)
    dist.barrier(torch)
    wall = time.perf_counter() - wall0
    ck = clocks.stop()
    per = [s.elapsed_time(e) / 1e3 for s, e in zip(starts, ends)]
    t_local = sum(per)
    t_max = dist.max(torch, t_local)
    st = pbh.sssp_stats(ws)
    units = dist.sum(torch, float(m_reached * args.steps))
    value = units / t_max / 1e9
    ms_step = 1e3 * t_max / args.steps
    peak, peak_kind = measured_peaks()
    ab = algorithmic_bytes(g.n, g.m, reached)
    achieved = ab / (t_local / args.steps) / 1e9
    # end to end through the host-buffer entry point (copies inside the region)
    e2e = None
    if args.e2e:
        hb = pbh.HostBuffers(g)
        hws = None
        for _ in range(max(1, args.warmup // 2)):
            _, hws = pbh.sssp_host(g, 0, r=r, d=d, cta=args.cta, ws=hws, pinned=hb, flags=flags)
        torch.cuda.synchronize()
        k = max(1, args.steps // 2)
        t0 = time.perf_counter()
        for _ in range(k):
            _, hws = pbh.sssp_host(g, 0, r=r, d=d, cta=args.cta, ws=hws, pinned=hb, flags=flags)
        te = (time.perf_counter() - t0) / k
        assert np.array_equal(hb.dist[: g.n], dist_host), "host entry point disagrees with the device one"
        e2e = {"value": m_reached / te / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": hb.h2d_bytes,
               "d2h_bytes_per_step": 8 * g.n, "ms_per_step": 1e3 * te}
    cfg.update({"r": st["r_eff"], "d": d or 65536, "team": "cta" if args.cta else "grid",
                "levels": st["levels"], "rounds": st["rounds"], "extracted": st["extracted"],
                "settle": bool(args.settle), "settled": st["settled"],
                "l2": "flushed between steps (256 MiB write outside the timed events)",
                "parallelism": f"replicas{dist.world}" if dist.world > 1 else "single"})
    out = {
        "metric": "SSSP GTEPS (single query, parDijkstra over the parallel bucket heap)",
        "value": value, "unit": "GTEPS", "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic", "config": cfg,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "traffic": committed_traffic(f"k_sssp_grid_banded_n2e{LOGN}_traffic.md")
                     if args.workload == "banded" and not args.cta else None,
                     "kernel": "k_sssp_grid" if not args.cta else "k_sssp_cta",
                     "algorithmic_bytes_per_launch": ab},
        "clocks": ck, "gpu_launches": args.steps, "wall_s": wall,
    }
    if e2e:
        out["e2e"] = e2e
    return out, g, m_reached


def cpu_oracle_sssp(g, source, m_reached, budget_s=20.0, max_runs=5):
    import oracle
    times = []
    t_all = time.perf_counter()
    while len(times) < max_runs and (time.perf_counter() - t_all) < budget_s:
        t0 = time.perf_counter()
        oracle.dijkstra(g, source)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    return {"value": m_reached / t / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
            "sample": f"full workload, {len(times)} run(s) of sequential binary-heap Dijkstra, median "
                      f"{t:.3f} s"}


# ------------------------------------------------------------ heap op stream

def bench_heap(args, dist: Dist, torch, pbh):
    key_space, d, batch, r = 1 << 24, 1 << 16, 1 << 16, 1 << 14
    rounds = args.rounds
    # record the stream with one untimed pass (the generator needs the
    # extracted keys of each round; they come from this device run)
    hs = gen.HeapStream(key_space, 2)
    h = pbh.Heap(key_space, d)
    keys, prios = [], []
    t0 = time.perf_counter()
    for _ in range(rounds):
        k, p = hs.next_batch(batch)
        kt = torch.from_numpy(k.view(np.int32)).cuda()
        pt = torch.from_numpy(p.view(np.int32)).cuda()
        keys.append(kt)
        prios.append(pt)
        h.bulk_update(kt, pt)
        ek, _ = h.extract_min(r)
        hs.observe_extracted(ek)
    h.sync()
    log(f"heap stream recorded in {time.perf_counter() - t0:.1f}s")
    del h
    # timed replay on a fresh heap
    reps = []
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(dist.local)
    for rep in range(args.warmup + args.steps):
        h = pbh.Heap(key_space, d)
        torch.cuda.synchronize()
        if rep == args.warmup:
            clocks.start()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for i in range(rounds):
            h.bulk_update(keys[i], prios[i])
            h.extract_min_async(r)
        e.record(stream)
        h.sync()
        if rep >= args.warmup:
            reps.append(s.elapsed_time(e) / 1e3)
        del h
    ck = clocks.stop()
    t = dist.max(torch, sum(reps))
    ops = (batch + r) * rounds * len(reps)
    value = dist.sum(torch, ops) / t
    cfg = {"workload": f"bucket-heap op stream: key space 2^24, {rounds} rounds of BulkUpdate(2^16 pairs) + "
                       f"extract_min(2^14), d=2^16", "rounds": rounds, "d": d}
    return {"metric": "heap ops/s (BulkUpdate elements + extracted elements per second)", "value": value,
            "unit": "ops/s", "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / len(reps), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic", "config": cfg, "clocks": ck,
            "gpu_launches": 2 * rounds * len(reps)}


def heap_general_stream(rounds, seed=3):
    """General-update op stream (open loop): every round pbh_assign of 2^16
    pairs with keys uniform over the 2^24 key space (later rounds mostly hit
    live keys, so priorities move up and down) and priorities uniform in
    [0, 2^32); pbh_delete of 2^12 keys uniform over the key space;
    extract_min(2^14)."""
    st = gen.Stream(seed)
    out = []
    for _ in range(rounds):
        ak = gen.uniform_u32(1 << 16, 0, (1 << 24) - 1, st.next())
        ap = gen.uniform_u32(1 << 16, 0, (1 << 32) - 1, st.next())
        dk = gen.uniform_u32(1 << 12, 0, (1 << 24) - 1, st.next())
        out.append((ak, ap, dk))
    return out


def cpu_oracle_heap_general(stream, r, budget_s=15.0):
    """The oracle (sorted-array queue) on the first rounds of the stream, as
    many as fit in budget_s seconds: (ops/s, rounds run)."""
    import oracle
    q = oracle.SortedPQ(1 << 24)
    ops, t = 0, 0.0
    done = 0
    for ak, ap, dk in stream:
        t0 = time.perf_counter()
        q.assign(ak, ap)
        q.delete(dk)
        q.extract_min(r)
        t += time.perf_counter() - t0
        ops += len(ak) + len(dk) + r
        done += 1
        if t > budget_s:
            break
    return ops / t, done


def bench_heap_general(args, dist: Dist, torch, pbh):
    key_space, d, r = 1 << 24, 1 << 16, 1 << 14
    rounds = args.rounds
    stream = heap_general_stream(rounds)
    dev = [(torch.from_numpy(a.view(np.int32)).cuda(), torch.from_numpy(p.view(np.int32)).cuda(),
            torch.from_numpy(k.view(np.int32)).cuda()) for a, p, k in stream]
    reps = []
    cur = torch.cuda.current_stream()
    clocks = ClockSampler(dist.local)
    for rep in range(args.warmup + args.steps):
        h = pbh.Heap(key_space, d)
        torch.cuda.synchronize()
        if rep == args.warmup:
            clocks.start()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(cur)
        for ak, ap, dk in dev:
            h.assign(ak, ap)
            h.delete(dk)
            h.extract_min_async(r)
        e.record(cur)
        h.sync()
        if rep >= args.warmup:
            reps.append(s.elapsed_time(e) / 1e3)
        live = h.size()
        del h
    ck = clocks.stop()
    t = dist.max(torch, sum(reps))
    per_round = (1 << 16) + (1 << 12) + r
    value = dist.sum(torch, per_round * rounds * len(reps)) / t
    cfg = {"workload": f"general heap op stream: key space 2^24, {rounds} rounds of assign(2^16 pairs, keys and "
                       f"priorities uniform: up and down) + delete(2^12 uniform keys) + extract_min(2^14), d=2^16",
           "rounds": rounds, "d": d, "live_at_end": live}
    res = {"metric": "heap ops/s (assign + delete + extracted elements per second)", "value": value,
           "unit": "ops/s", "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": 1e3 * t / len(reps), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "u64", "data": "synthetic", "config": cfg, "clocks": ck,
           "gpu_launches": 3 * rounds * len(reps)}
    if args.cpu and dist.rank == 0:
        v, done = cpu_oracle_heap_general(stream, r)
        res["cpu_baseline"] = {"value": v, "unit": "ops/s", "cores": 1, "kind": "oracle",
                               "sample": f"the first {done} rounds of the same stream (small live set: the "
                                         f"oracle slows as it grows)"}
    return res


# ------------------------------------------------------------ batched queries

def batch_queries(nq=512, seed=4):
    """512 SSSP queries on graphs of uneven size: half square grids with side
    2^U(5,9) (32x32 .. 512x512), half banded graphs with n = 2^U(12,18),
    degree U{16..64} and window +-256; weights uniform in [1, 65535]; graph q
    seeded 1000 + q; source uniform."""
    st = gen.Stream(seed)
    graphs, sources = [], []
    for q in range(nq):
        if q % 2 == 0:
            side = int(round(2 ** (5 + 4 * st.random())))
            g = gen.grid(side, side, 1, 65535, 1000 + q)
        else:
            n = int(round(2 ** (12 + 6 * st.random())))
            g = gen.banded(n, st.uniform(16, 64), 256, 1, 65535, 1000 + q)
        graphs.append(g)
        sources.append(st.uniform(0, g.n - 1))
    return graphs, sources


def bench_batch(args, dist: Dist, torch, pbh):
    from paper_1908_09378_gb300 import autotune
    t0 = time.perf_counter()
    graphs, sources = batch_queries(args.queries)
    # queries are independent: each rank takes its share, no collective on the data path
    mine = shard([g.n + g.m for g in graphs], dist.rank, dist.world)
    graphs = [graphs[i] for i in mine]
    sources = [sources[i] for i in mine]
    log(f"rank {dist.rank}: {len(graphs)} graphs generated in {time.perf_counter() - t0:.1f}s, "
        f"m total {sum(g.m for g in graphs) / 1e6:.1f}M")
    dgs = [pbh.DeviceGraph(g) for g in graphs]
    rs, ds = autotune.batch_params(dgs)
    b = pbh.Batch(dgs, sources, r=rs, d=ds)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        b.run_async()
        code, st, rounds = b.status()
        if code != 0:
            bad = [(i, s & 0xFFFF, s >> 16, graphs[i].n, rs[i], ds[i]) for i, s in enumerate(st) if s]
            raise RuntimeError(f"batch failed: (query, status, site, n, r, d) {bad[:20]}")
    m_reached = 0
    for g, dd in zip(graphs, b.dist):
        dh = dd[: g.n].cpu().numpy().view(np.uint64)
        deg = np.diff(g.row_ptr.astype(np.int64))
        m_reached += int(deg[dh != np.uint64(0xFFFFFFFFFFFFFFFF)].sum())
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    clocks = ClockSampler(dist.local)
    clocks.start()
    per = []
    for i in range(args.steps):
        flush.fill_(i)
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        b.run_async()
        e.record(stream)
        torch.cuda.synchronize()
        per.append(s.elapsed_time(e) / 1e3)
    ck = clocks.stop()
    t = dist.max(torch, sum(per))
    qps = dist.sum(torch, len(graphs) * args.steps) / t
    # the one-query-at-a-time plain path on the same queries (sssp_run, whole GPU each)
    ws = {}
    one = []
    for rep in range(2):
        t1 = time.perf_counter()
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for dg, src in zip(dgs, sources):
            key = dg.n
            if key not in ws:
                ws[key] = pbh.SsspWorkspace(dg.n)
            pbh.sssp_async(dg, src, ws=ws[key])
        e.record(stream)
        torch.cuda.synchronize()
        one.append(s.elapsed_time(e) / 1e3)
    t_one = min(one)
    qps_one = len(graphs) / t_one
    cfg = {"workload": f"{args.queries} SSSP queries: half square grids side 2^U(5,9), half banded n=2^U(12,18) "
                       "deg U{16..64} window +-256, w~U[1,65535], graph q seeded 1000+q, uniform sources",
           "queries": args.queries, "queries_this_rank": len(graphs), "team": "one CTA per query",
           "parallelism": f"queries sharded over {dist.world} GPU(s), no collective" ,
           "params": autotune.describe(), "l2": "flushed between steps (256 MiB write outside the timed events)"}
    return {"metric": "batched SSSP queries/s (one persistent launch)", "value": qps, "unit": "queries/s",
            "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": cfg, "gteps_aggregate": dist.sum(torch, m_reached * args.steps) / t / 1e9,
            "one_at_a_time": {"value": qps_one, "unit": "queries/s", "ms": 1e3 * t_one,
                              "path": "sssp_run per query, whole-GPU cooperative grid, default options"},
            "speedup_vs_one_at_a_time": qps / qps_one, "clocks": ck, "gpu_launches": args.steps}


# ------------------------------------------------------------ served queries

def serve_pool(seed=6):
    """Resident graph pool: 32 square grids with n = 2^U(10,20) and 32 banded
    graphs with n = 2^U(12,20), degree 32, window +-256; weights uniform in
    [1, 65535]; graph g seeded 2000 + g."""
    st = gen.Stream(seed)
    graphs = []
    for q in range(64):
        if q < 32:
            side = int(round(2 ** ((10 + 10 * st.random()) / 2)))
            graphs.append(gen.grid(side, side, 1, 65535, 2000 + q))
        else:
            n = int(round(2 ** (12 + 8 * st.random())))
            graphs.append(gen.banded(n, 32, 256, 1, 65535, 2000 + q))
    return graphs


def serve_requests(graphs, n, rate, seed):
    from paper_1908_09378_gb300.serve import poisson_arrivals
    st = gen.Stream(seed + 17)
    reqs = []
    for a in poisson_arrivals(n, rate, seed):
        gi = st.uniform(0, len(graphs) - 1)
        reqs.append((a, gi, st.uniform(0, graphs[gi].n - 1)))
    return reqs


def bench_serve(args, dist: Dist, torch, pbh):
    from paper_1908_09378_gb300 import serve
    t0 = time.perf_counter()
    graphs = serve_pool()
    dgs = [pbh.DeviceGraph(g) for g in graphs]
    log(f"pool of {len(graphs)} graphs, m total {sum(g.m for g in graphs) / 1e6:.1f}M, "
        f"generated in {time.perf_counter() - t0:.1f}s")
    budget = 40 << 30
    sv = serve.Server(budget_bytes=budget, slots=32768)
    try:
        # warm-up and capacity C: a burst of requests all arriving at t = 0
        serve.run_stream(sv, dgs, serve_requests(graphs, 500, 0.0, 1))
        burst = serve.run_stream(sv, dgs, serve_requests(graphs, 4000, 0.0, 2))
        cap = burst["qps"]
        clocks = ClockSampler(dist.local)
        clocks.start()
        lat = serve.run_stream(sv, dgs, serve_requests(graphs, args.requests, 0.8 * cap, 3))
        sat = serve.run_stream(sv, dgs, serve_requests(graphs, args.requests, 2.0 * cap, 4))
        ck = clocks.stop()
    finally:
        sv.stop()
    # one-query-at-a-time plain path on a sample of the same stream
    sample = serve_requests(graphs, 200, 0.0, 4)
    ws = {}
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _, gi, src in sample:
        dg = dgs[gi]
        if dg.n not in ws:
            ws[dg.n] = pbh.SsspWorkspace(dg.n)
        pbh.sssp_async(dg, src, ws=ws[dg.n])
    torch.cuda.synchronize()
    qps_one = len(sample) / (time.perf_counter() - t1)
    cfg = {"workload": f"Poisson stream of {args.requests} SSSP queries over a resident pool of 32 grids "
                       "(n 2^10..2^20) and 32 banded graphs (n 2^12..2^20, degree 32, window +-256), "
                       "w~U[1,65535]; uniform graph and source", "requests": args.requests,
           "budget_bytes": budget, "capacity_qps": cap, "rate_latency_run": 0.8 * cap,
           "rate_saturated_run": 2.0 * cap, "team": "one CTA per query, one persistent launch"}
    return {"metric": "served SSSP queries/s (continuous batching) and p50/p99 latency", "value": sat["qps"],
            "unit": "queries/s", "n_gpus": dist.world, "steps": 1, "warmup": 1,
            "ms_per_step": 1e3 * sat["wall_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": cfg,
            "latency": {"p50_ms": lat["p50_ms"], "p99_ms": lat["p99_ms"], "mean_ms": lat["mean_ms"],
                        "qps": lat["qps"], "device_p50_ms": lat["device_p50_ms"]},
            "saturated": sat, "peak_pool_bytes": max(lat["peak_pool_bytes"], sat["peak_pool_bytes"]),
            "one_at_a_time": {"value": qps_one, "unit": "queries/s", "sample": len(sample)},
            "speedup_vs_one_at_a_time": sat["qps"] / qps_one, "clocks": ck, "gpu_launches": 3}


# ------------------------------------------------------------ reference arm

def reference_arm(args):
    """The CPU oracle, as it stands, on the same workload and metric."""
    import oracle
    if args.workload not in ("banded", "grid64"):
        return {"impl": "reference", "unavailable": f"no oracle arm for workload {args.workload}"}
    g = banded_graph() if args.workload == "banded" else gen.grid(64, 64, 1, 100, 0)
    cfg = banded_cfg() if args.workload == "banded" else {"workload": "64x64 grid", "n": g.n, "m": g.m}
    d0 = oracle.dijkstra(g, 0)
    deg = np.diff(g.row_ptr.astype(np.int64))
    m_reached = int(deg[d0 != oracle.INF].sum())
    for _ in range(args.warmup):
        oracle.dijkstra(g, 0)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.dijkstra(g, 0)
        times.append(time.perf_counter() - t0)
    t = sum(times)
    value = m_reached * args.steps / t / 1e9
    sample = f"full workload per step: sequential binary-heap Dijkstra from source 0 ({args.steps} steps)"
    return {"impl": "reference", "metric": "SSSP GTEPS (single query, parDijkstra over the parallel bucket heap)",
            "value": value, "unit": "GTEPS", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------ main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="banded", choices=["banded", "grid64", "dag", "heap", "heap_general", "batch",
                                                           "serve"])
    ap.add_argument("--m", type=int, default=100_000_000, help="dag workload: arcs")
    ap.add_argument("--requests", type=int, default=20000, help="serve workload: requests per run")
    ap.add_argument("--queries", type=int, default=512, help="batch workload: number of queries")
    ap.add_argument("--r", type=int, default=0, help="extract width (0 = library default)")
    ap.add_argument("--d", type=int, default=0, help="heap parameter d (0 = library default)")
    ap.add_argument("--cta", type=int, default=0, help="1 = one-CTA team instead of the whole GPU")
    ap.add_argument("--settle", action="store_true", help="single-query workloads: the settle criterion flag")
    ap.add_argument("--rounds", type=int, default=1000, help="heap workload rounds")
    ap.add_argument("--n", type=int, default=20, help="log2 vertices of the banded workload (profiling only)")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu", action="store_false")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    global LOGN
    LOGN = args.n

    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return 0
        print(json.dumps(reference_arm(args)), flush=True)
        return 0

    import torch
    import paper_1908_09378_gb300 as pbh
    pbh.load()
    dist = Dist(args.gpus)
    dist.init(torch)
    if args.workload == "heap":
        out = bench_heap(args, dist, torch, pbh)
    elif args.workload == "heap_general":
        out = bench_heap_general(args, dist, torch, pbh)
    elif args.workload == "batch":
        out = bench_batch(args, dist, torch, pbh)
    elif args.workload == "serve":
        out = bench_serve(args, dist, torch, pbh)
    else:
        out, g, m_reached = bench_sssp(args, dist, torch, pbh)
        if args.cpu and dist.rank == 0:
            out["cpu_baseline"] = cpu_oracle_sssp(g, 0, m_reached)
    if dist.rank == 0:
        print(json.dumps(out), flush=True)
    dist.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
