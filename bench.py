#!/usr/bin/env python3
"""Benchmark of parDijkstra and the GB300 parallel bucket heap.

Default run (one JSON line, rank 0): the headline is single-source shortest
paths on the banded high-diameter graph (n = 2^20 vertices, 64 distinct
out-arcs per vertex drawn uniformly from [i-512, i+512], m = 2^26 arcs,
uint32 weights uniform in [1, 65535], seed 1, source 0).  One step = one
complete sssp_run (all rounds of extract-min / relax / BulkUpdate, on the
device) with the graph resident in HBM; metric GTEPS = reached arcs / time.
The line also carries, under "configs", the other four workloads, each with
its own metric, roofline, CPU baseline and a check against the oracle made
outside the timed region:
  grid64  the 64x64 grid (GTEPS),
  heap    the bucket-heap op stream: key space 2^24, 1000 rounds of
          BulkUpdate(2^16 pairs) + extract_min(2^14) (heap ops/s),
  batch   512 mixed queries in one persistent launch (queries/s),
  serve   a Poisson stream of 20k queries through the persistent server
          (queries/s, p50/p99 latency).

--workload runs one workload alone (banded, grid64, dag, heap, heap_general,
batch, serve).  --impl reference times the CPU oracle on the headline
workload instead (the one place besides the CPU-baseline legs where this
script runs oracle/ code).  --gpus N without a torchrun environment starts N
ranks itself.
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
from concurrent.futures import ThreadPoolExecutor

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


def kernel_source_hash(unit: str = None) -> str:
    """Hash of the CUDA sources a committed ncu traffic figure was taken on:
    with `unit` (a .cu file of csrc/), that translation unit, i.e. the file
    and every header of csrc/ it includes, directly or not; without it, every
    source.  A figure is used only while its kernel's sources are unchanged."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_1908_09378_gb300", "csrc")
    names = sorted(n for n in os.listdir(csrc) if n.endswith((".cu", ".cuh", ".h")))
    if unit is not None:
        todo, seen = [unit], set()
        while todo:
            name = todo.pop()
            if name in seen or name not in names:
                continue
            seen.add(name)
            with open(os.path.join(csrc, name)) as f:
                todo += re.findall(r'^\s*#\s*include\s+"([^"]+)"', f.read(), flags=re.M)
        if unit not in seen:
            raise FileNotFoundError(f"no translation unit {unit} in csrc/")
        names = sorted(seen)
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def tuned_table_hash() -> str:
    """Hash of the autotuner's table (the batch's per-query parameters)."""
    import hashlib
    p = os.path.join(ROOT, "paper_1908_09378_gb300", "tuned.json")
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16] if os.path.exists(p) else "none"


def committed_traffic(profile_name: str, params: str = None):
    """Bytes per launch from a profiles/ summary, or None: only while the
    sources of the captured kernel's translation unit (its `kernel_unit`
    line) hash to the recorded value and, with params, the launch parameters
    the capture was taken with are the same."""
    p = os.path.join(ROOT, "profiles", profile_name)
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line and line.strip().startswith(("traffic_bytes_per_launch", "kernel_source_hash",
                                                    "kernel_unit", "launch_params")):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if "traffic_bytes_per_launch" not in vals or vals.get("kernel_source_hash") != kernel_source_hash(
            vals.get("kernel_unit")):
        return None
    if params is not None and vals.get("launch_params") != params:
        return None
    return int(vals["traffic_bytes_per_launch"])


def cpu_model() -> str:
    """The host CPU's model name (for the CPU baselines)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1


def par_map(fn, items, threads=None):
    """fn over items on a thread pool (the C generators and the oracle release
    the GIL inside their calls), results in order."""
    items = list(items)
    threads = threads or host_cores()
    if threads <= 1 or len(items) <= 1:
        return [fn(x) for x in items]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(fn, items))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------ workloads

LOGN = 20  # banded workload size (the benchmark line is quoted at 2^20; smaller only for profiling)
GOLDEN = os.path.join(ROOT, "tests", "golden")


def banded_graph(logn=None):
    logn = LOGN if logn is None else logn
    return gen.banded(1 << logn, 64, 512, 1, 65535, 1)


def banded_cfg(logn=None):
    logn = LOGN if logn is None else logn
    return {"workload": f"banded n=2^{logn}, 64 distinct out-arcs in [i-512,i+512], m=2^{logn + 6}, "
                        "w~U[1,65535] (seed 1), source 0", "n": 1 << logn, "m": 1 << (logn + 6)}


def stored_counts(name: str):
    """The oracle's counts for a benchmark graph from tests/golden/relaxations.txt
    (written by tests/golden/make_relaxations.py, which calls only the oracle):
    dict(n, m, reached, reached_arcs, U), or None."""
    path = os.path.join(GOLDEN, "relaxations.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if f and f[0] == name:
            n, m, reached, arcs, U = (int(x) for x in f[1:6])
            return {"n": n, "m": m, "reached": reached, "reached_arcs": arcs, "U": U}
    return None


def algorithmic_bytes(n: int, m_read: int, U: int) -> int:
    """Bytes one SSSP query must move once: the row pointers (8(n+1)), the
    column and weight arrays of the arcs it scans (8 per arc), the distance
    write (8n) and one heap word written and read per successful relaxation
    of the oracle's r = 1 run (16 U)."""
    return 8 * (n + 1) + 8 * m_read + 8 * n + 16 * U


def reached_arcs(g, dist_host) -> int:
    deg = np.diff(g.row_ptr.astype(np.int64))
    return int(deg[dist_host != np.uint64(0xFFFFFFFFFFFFFFFF)].sum())


def roofline(ab: int, seconds_per_launch: float, kernel: str, traffic=None, **extra):
    peak, peak_kind = measured_peaks()
    achieved = ab / seconds_per_launch / 1e9
    out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "peak_kind": peak_kind, "traffic": traffic, "kernel": kernel, "algorithmic_bytes_per_launch": ab}
    out.update(extra)
    return out


def single_workload(name: str, m_dag: int = 100_000_000):
    """(graph, config, stored-count name) of a single-query workload."""
    if name == "banded":
        return banded_graph(), banded_cfg(), f"banded_n2e{LOGN}"
    if name == "dag":
        g = gen.dag(30000, m_dag, 0)
        return g, {"workload": f"the paper's random DAG (Section 4.2): n=30000, m={g.m}, chain of weight 1 plus "
                               "forward arcs of weight 2(v-u), seed 0, source 0", "n": g.n, "m": g.m}, None
    g = gen.grid(64, 64, 1, 100, 0)
    return g, {"workload": "64x64 directed 4-neighbour grid, m=16128, w~U[1,100] (seed 0), source 0",
               "n": g.n, "m": g.m}, "grid64"


def bench_sssp(args, dist: Dist, torch, pbh, workload: str, steps: int, warmup: int, e2e: bool, cpu: bool):
    g, cfg, counts_name = single_workload(workload, args.m)
    dg = pbh.DeviceGraph(g)
    r, d, cta = args.r, args.d, args.cta
    tuned = None
    if workload == "dag":
        r = r or 1                              # the paper's parDijkstra: one vertex per round
        d = d or max(1, r) * dg.max_degree      # d = maximum degree (Section 4.1)
    elif not (r or d or cta or args.settle):
        # the autotuned team, r and d of this size class
        from paper_1908_09378_gb300 import autotune
        cta, r, d = autotune.single_params(g.n, g.m, dg.max_degree)
        tuned = autotune.describe_single(g.n, dg.max_degree)
    args_cta = cta
    flags = pbh.SSSP_SETTLE if args.settle else 0
    ws = pbh.SsspWorkspace(dg.n, r, d, cta, flags=flags)
    distv = torch.empty(dg.n, dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        pbh.sssp_async(dg, 0, dist=distv, ws=ws)
    pbh.sssp_stats(ws)
    dist_host = distv.cpu().numpy().view(np.uint64)
    reached = int((dist_host != np.uint64(0xFFFFFFFFFFFFFFFF)).sum())
    m_reached = reached_arcs(g, dist_host)
    # timed: one event pair per step on the launching stream, L2 flushed between steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    clocks = ClockSampler(dist.local)
    dist.barrier(torch)
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(steps):
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
    units = dist.sum(torch, float(m_reached * steps))
    value = units / t_max / 1e9
    # the oracle: distances checked element by element, U counted (rank 0)
    cpu_base, check, U = None, None, None
    sc = stored_counts(counts_name) if counts_name else None
    if cpu and dist.rank == 0:
        cpu_base, want, U = cpu_oracle_sssp(g, 0, m_reached)
        check = {"compared": "every vertex", "mismatches": int((want != dist_host).sum())}
        if check["mismatches"]:
            raise RuntimeError(f"{workload}: {check['mismatches']} distances differ from the oracle")
        if sc and sc["U"] != U:
            raise RuntimeError(f"{workload}: stored U {sc['U']} differs from the oracle's {U}")
    elif sc:
        U = sc["U"]
    ab = algorithmic_bytes(g.n, m_reached, U) if U is not None else None
    e2e_out = None
    if e2e:
        # end to end through the host-buffer entry point (copies inside the region)
        hb = pbh.HostBuffers(g)
        hws = None
        for _ in range(max(1, warmup // 2)):
            _, hws = pbh.sssp_host(g, 0, r=r, d=d, cta=args_cta, ws=hws, pinned=hb, flags=flags)
        torch.cuda.synchronize()
        k = max(1, steps // 2)
        t0 = time.perf_counter()
        for _ in range(k):
            _, hws = pbh.sssp_host(g, 0, r=r, d=d, cta=args_cta, ws=hws, pinned=hb, flags=flags)
        te = (time.perf_counter() - t0) / k
        if not np.array_equal(hb.dist[: g.n], dist_host):
            raise RuntimeError("host entry point disagrees with the device one")
        e2e_out = {"value": m_reached / te / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": hb.h2d_bytes,
                   "d2h_bytes_per_step": 8 * g.n, "ms_per_step": 1e3 * te}
    team = ("grid" if args_cta == 0 else "cta" if args_cta == 1 else
            f"cluster{args_cta}" if args_cta <= 16 else f"grid of {args_cta} CTAs")
    cfg.update({"r": st["r_eff"], "d": d or 65536, "team": team, "params": tuned or "given on the command line",
                "levels": st["levels"], "rounds": st["rounds"], "extracted": st["extracted"],
                "settle": bool(args.settle), "settled": st["settled"],
                "l2": "flushed between steps (256 MiB write outside the timed events)",
                "parallelism": f"replicas{dist.world}" if dist.world > 1 else "single"})
    kernel = "k_sssp_cta" if args_cta == 1 else "k_sssp_cluster" if 2 <= args_cta <= 16 else "k_sssp_grid"
    traffic = (committed_traffic(f"k_sssp_grid_banded_n2e{LOGN}_traffic.md", f"r={st['r_eff']} d={d or 65536}")
               if workload == "banded" and kernel == "k_sssp_grid" else None)
    out = {
        "metric": "SSSP GTEPS (single query, parDijkstra over the parallel bucket heap)",
        "value": value, "unit": "GTEPS", "n_gpus": dist.world, "steps": steps, "warmup": warmup,
        "ms_per_step": 1e3 * t_max / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic", "config": cfg,
        "roofline": roofline(ab, t_local / steps, kernel, traffic, U=U, bytes_formula="8(n+1) + 8 m_reached + 8n + 16U")
        if ab else None,
        "clocks": ck, "gpu_launches": steps, "wall_s": wall,
        "us_per_round": 1e6 * t_local / steps / max(st["rounds"], 1),
    }
    if e2e_out:
        out["e2e"] = e2e_out
    if cpu_base:
        out["cpu_baseline"] = cpu_base
        out["oracle_check"] = check
    return out


def cpu_oracle_sssp(g, source, m_reached, budget_s=20.0, max_runs=5):
    """The oracle (sequential binary-heap Dijkstra) on one host core:
    (cpu_baseline, its distances, its successful relaxations U)."""
    import oracle
    times = []
    want = U = None
    t_all = time.perf_counter()
    while len(times) < max_runs and (time.perf_counter() - t_all) < budget_s:
        t0 = time.perf_counter()
        d, _, _, u = oracle.dijkstra_counts(g, source)
        times.append(time.perf_counter() - t0)
        want, U = d, u
    t = statistics.median(times)
    return ({"value": m_reached / t / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle", "cpu": cpu_model(),
             "sample": f"full workload, {len(times)} run(s) of sequential binary-heap Dijkstra, median {t:.3f} s"},
            want, U)


# ------------------------------------------------------------ heap op stream

HEAP_BYTES_PER_ROUND = 8 * (1 << 16) + 8 * (1 << 14) + 16 * (1 << 16)


def bench_heap(args, dist: Dist, torch, pbh, rounds: int, steps: int, warmup: int, cpu: bool):
    """The heap op stream.  An untimed pass records the closed-loop stream on the
    device (the generator learns which keys left from each extract) and, on
    rank 0, compares the first rounds op by op with the oracle, timing the
    oracle on them (the CPU baseline); then the recorded stream is replayed
    on fresh heaps with CUDA events around each replay."""
    key_space, d, batch, r = 1 << 24, 1 << 16, 1 << 16, 1 << 14
    hs = gen.HeapStream(key_space, 2)
    h = pbh.Heap(key_space, d)
    q = None
    if cpu and dist.rank == 0:
        import oracle
        q = oracle.SortedPQ(key_space)
    keys, prios = [], []
    cpu_keys = []
    t_cpu, cpu_rounds, mismatches = 0.0, 0, 0
    t0 = time.perf_counter()
    for i in range(rounds):
        k, p = hs.next_batch(batch)
        kt = torch.from_numpy(k.view(np.int32)).cuda()
        pt = torch.from_numpy(p.view(np.int32)).cuda()
        keys.append(kt)
        prios.append(pt)
        h.bulk_update(kt, pt)
        ek, ep = h.extract_min(r)
        if q is not None and t_cpu < args.cpu_budget:
            c0 = time.perf_counter()
            q.bulk_update(k, p)
            wk, wp = q.extract_min(r)
            t_cpu += time.perf_counter() - c0
            cpu_rounds += 1
            cpu_keys.append(wk)
            mismatches += int(not (np.array_equal(ek, wk) and np.array_equal(ep, wp)))
        hs.observe_extracted(ek)
    h.sync()
    log(f"heap stream recorded in {time.perf_counter() - t0:.1f}s ({cpu_rounds} rounds compared with the oracle)")
    if mismatches:
        raise RuntimeError(f"heap: {mismatches} of {cpu_rounds} rounds differ from the oracle")
    del h
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(dist.local)
    merged = None
    # the recorded stream as one operation sequence (pbh_run_ops); outputs reused
    seq_ops = []
    for i in range(rounds):
        seq_ops += [("bulk", keys[i], prios[i]), ("extract", r)]
    seq_outs = None

    def replay(path):
        nonlocal merged, seq_outs
        h = pbh.Heap(key_space, d)
        arr = None
        if path != "per_operation":
            arr, seq_outs, keep = h.ops_array(seq_ops, seq_outs)
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        if path == "per_operation":
            for i in range(rounds):
                h.bulk_update(keys[i], prios[i])
                h.extract_min_async(r)
        else:
            h.run_ops(seq_ops, deep_ctas=args.deep_ctas if path == "sequence_concurrent" else 0, outs=seq_outs,
                      arr=arr)
        e.record(stream)
        h.sync()
        if merged is None:
            merged = h.stats()["merged"]
        del h
        return s.elapsed_time(e) / 1e3

    paths = {}
    clocks.start()
    for path in ("per_operation", "sequence_phase_by_phase", "sequence_concurrent"):
        reps = [replay(path) for _ in range(warmup + steps)][warmup:]
        paths[path] = reps
    ck = clocks.stop()
    best = min(paths, key=lambda p: sum(paths[p]))
    reps = paths[best]
    t_local = sum(reps)
    t = dist.max(torch, t_local)
    ops = (batch + r) * rounds * len(reps)
    value = dist.sum(torch, ops) / t
    launches = 2 * rounds if best == "per_operation" else (2 * rounds + 4095) // 4096
    ab = (HEAP_BYTES_PER_ROUND * rounds + 16 * merged) // launches
    cfg = {"workload": f"bucket-heap op stream: key space 2^24, {rounds} rounds of BulkUpdate(2^16 pairs) + "
                       f"extract_min(2^14), d=2^16, seed 2, closed loop", "rounds": rounds, "d": d,
           "inputs": "recorded batches (512 MiB > L2) replayed on a fresh heap per step", "path": best,
           "deep_ctas": args.deep_ctas}
    out = {"metric": "heap ops/s (BulkUpdate elements + extracted elements per second)", "value": value,
           "unit": "ops/s", "n_gpus": dist.world, "steps": steps, "warmup": warmup,
           "ms_per_step": 1e3 * t / len(reps), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "u64", "data": "synthetic", "config": cfg, "clocks": ck, "gpu_launches": launches * len(reps),
           "paths": {p: {"ops_per_s": (batch + r) * rounds * len(v) / sum(v), "ms_per_step": 1e3 * sum(v) / len(v)}
                     for p, v in paths.items()},
           "roofline": roofline(ab, t_local / len(reps) / launches, "k_pbh_op" if best == "per_operation" else
                                "k_pbh_ops", None, merged_per_step=merged,
                                bytes_formula="per round 8*2^16 read + 8*2^14 written + 16*2^16 cur RMW; "
                                              "plus 16 per element merged by a Resolve, over the launches")}
    if seq_outs is not None:
        # the sequence's extracts against the oracle's rounds compared above
        n_cmp = min(cpu_rounds, rounds)
        for i in range(n_cmp):
            ko, po, co = seq_outs[i]
            n = int(co.item())
            gk = ko[:n].cpu().numpy().view(np.uint32)
            if i < len(cpu_keys) and not np.array_equal(gk, cpu_keys[i]):
                raise RuntimeError(f"heap sequence: extract {i} differs from the oracle")
    if q is not None:
        out["cpu_baseline"] = {"value": cpu_rounds * (batch + r) / t_cpu, "unit": "ops/s", "cores": 1,
                               "kind": "oracle", "cpu": cpu_model(),
                               "sample": f"the first {cpu_rounds} rounds of the same stream on the sorted-array "
                                         f"queue (about {args.cpu_budget:.0f} s; it slows as the live set grows)"}
        out["oracle_check"] = {"compared": f"extract output of the first {cpu_rounds} rounds, op by op",
                               "mismatches": mismatches}
    return out


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
        res["cpu_baseline"] = {"value": v, "unit": "ops/s", "cores": 1, "kind": "oracle", "cpu": cpu_model(),
                               "sample": f"the first {done} rounds of the same stream (small live set: the "
                                         f"oracle slows as it grows)"}
    return res


# ------------------------------------------------------------ batched queries

def batch_specs(nq=512, seed=4):
    """512 SSSP queries on graphs of uneven size: half square grids with side
    2^U(5,9) (32x32 .. 512x512), half banded graphs with n = 2^U(12,18),
    degree U{16..64} and window +-256; weights uniform in [1, 65535]; graph q
    seeded 1000 + q; source uniform.  Returns (kind, size, degree, seed,
    source) per query; the draws come from one stream in query order."""
    st = gen.Stream(seed)
    specs = []
    for q in range(nq):
        if q % 2 == 0:
            side = int(round(2 ** (5 + 4 * st.random())))
            specs.append(("grid", side, 4, 1000 + q, st.uniform(0, side * side - 1)))
        else:
            n = int(round(2 ** (12 + 6 * st.random())))
            deg = st.uniform(16, 64)
            specs.append(("banded", n, deg, 1000 + q, st.uniform(0, n - 1)))
    return specs


def make_spec_graph(spec):
    kind, size, deg, seed, _ = spec
    if kind == "grid":
        return gen.grid(size, size, 1, 65535, seed)
    return gen.banded(size, deg, 256, 1, 65535, seed)


def batch_queries(nq=512, seed=4, indices=None):
    specs = batch_specs(nq, seed)
    idx = range(nq) if indices is None else indices
    graphs = par_map(make_spec_graph, [specs[i] for i in idx])
    return graphs, [specs[i][4] for i in idx]


def oracle_pool(graphs, sources, threads=None):
    """The oracle on every (graph, source) on a thread pool of all host
    cores: (list of (dist, U), seconds, threads)."""
    import oracle
    threads = threads or host_cores()
    t0 = time.perf_counter()
    res = par_map(lambda gs: (lambda r: (r[0], r[3]))(oracle.dijkstra_counts(gs[0], gs[1])),
                  list(zip(graphs, sources)), threads)
    return res, time.perf_counter() - t0, threads


def bench_batch(args, dist: Dist, torch, pbh, steps: int, warmup: int, cpu: bool):
    """The batched queries: the queries of this rank in one persistent launch per step."""
    from paper_1908_09378_gb300 import autotune
    t0 = time.perf_counter()
    specs = batch_specs(args.queries)
    weights = [(s[1] * s[1] * 5 if s[0] == "grid" else s[1] * (s[2] + 1)) for s in specs]
    mine = shard(weights, dist.rank, dist.world)   # queries are independent: no collective on the data path
    graphs, sources = batch_queries(args.queries, indices=mine)
    log(f"rank {dist.rank}: {len(graphs)} graphs generated in {time.perf_counter() - t0:.1f}s, "
        f"m total {sum(g.m for g in graphs) / 1e6:.1f}M")
    dgs = [pbh.DeviceGraph(g) for g in graphs]
    rs, ds, cs = autotune.batch_params(dgs)
    b = pbh.Batch(dgs, sources, r=rs, d=ds, cta=cs)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        b.run_async()
        code, st, rounds = b.status()
        if code != 0:
            bad = [(i, s & 0xFFFF, s >> 16, graphs[i].n, rs[i], ds[i]) for i, s in enumerate(st) if s]
            raise RuntimeError(f"batch failed: (query, status, site, n, r, d) {bad[:20]}")
    got = [dd[: g.n].cpu().numpy().view(np.uint64) for g, dd in zip(graphs, b.dist)]
    m_reached = sum(reached_arcs(g, dh) for g, dh in zip(graphs, got))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    clocks = ClockSampler(dist.local)
    clocks.start()
    per = []
    for i in range(steps):
        flush.fill_(i)
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        b.run_async()
        e.record(stream)
        torch.cuda.synchronize()
        per.append(s.elapsed_time(e) / 1e3)
    ck = clocks.stop()
    code, st, rounds = b.status()
    if code != 0:
        raise RuntimeError(f"batch failed in the timed steps: {[s for s in st if s][:10]}")
    t_local = sum(per)
    t = dist.max(torch, t_local)
    qps = dist.sum(torch, len(graphs) * steps) / t
    # the one-query-at-a-time plain path on the same queries (sssp_run, whole GPU each)
    wss = {}
    one = []
    for rep in range(2):
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for dg, src in zip(dgs, sources):
            if dg.n not in wss:
                wss[dg.n] = pbh.SsspWorkspace(dg.n)
            pbh.sssp_async(dg, src, ws=wss[dg.n])
        e.record(stream)
        torch.cuda.synchronize()
        one.append(s.elapsed_time(e) / 1e3)
    t_one = min(one)
    qps_one = dist.sum(torch, len(graphs)) / dist.max(torch, t_one)
    # every query of this rank against the oracle (all host cores), which also
    # gives each query's U for the roofline and the CPU baseline
    res, t_cpu, threads = oracle_pool(graphs, sources)
    mism = [i for i, ((want, _), g) in enumerate(zip(res, got)) if not np.array_equal(want, g)]
    if mism:
        raise RuntimeError(f"batch: queries {mism[:10]} differ from the oracle")
    ab = sum(algorithmic_bytes(g.n, reached_arcs(g, dh), U) for g, dh, (_, U) in zip(graphs, got, res))
    cfg = {"workload": f"{args.queries} SSSP queries: half square grids side 2^U(5,9), half banded n=2^U(12,18) "
                       "deg U{16..64} window +-256, w~U[1,65535], graph q seeded 1000+q, uniform sources",
           "queries": args.queries, "queries_this_rank": len(graphs),
           "team": f"{sum(1 for c in cs if c >= 2)} queries on {max(cs)}-CTA clusters, the rest one CTA each"
           if max(cs) >= 2 else "one CTA per query",
           "parallelism": f"queries sharded over {dist.world} GPU(s), no collective",
           "params": autotune.describe(), "l2": "flushed between steps (256 MiB write outside the timed events)"}
    out = {"metric": "batched SSSP queries/s (one persistent launch)", "value": qps, "unit": "queries/s",
           "n_gpus": dist.world, "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * t / steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
           "config": cfg, "gteps_aggregate": dist.sum(torch, m_reached * steps) / t / 1e9,
           "roofline": roofline(ab, t_local / steps, "k_sssp_batch",
                                committed_traffic("k_sssp_batch_batch512_launch_list.md", tuned_table_hash())
                                if args.queries == 512 else None,
                                bytes_formula="sum over queries of 8(n+1) + 8 m_reached + 8n + 16U",
                                per="step (k_sssp_batch beside k_sssp_batch_cluster)"),
           "one_at_a_time": {"value": qps_one, "unit": "queries/s", "ms": 1e3 * t_one,
                             "path": "sssp_run per query, whole-GPU cooperative grid, default options"},
           "speedup_vs_one_at_a_time": qps / qps_one, "clocks": ck,
           # one launch per cluster size in use plus the one-CTA launch
           "gpu_launches": steps * (len({c for c in cs if c >= 2}) + (1 if any(c < 2 for c in cs) else 0)),
           "oracle_check": {"compared": f"all {len(graphs)} queries of this rank, every vertex", "mismatches": 0}}
    if dist.rank == 0 and cpu:
        out["cpu_baseline"] = {"value": len(graphs) / t_cpu, "unit": "queries/s", "cores": threads,
                               "kind": "oracle", "cpu": cpu_model(),
                               "sample": f"the same {len(graphs)} queries, sequential Dijkstra per query on a "
                                         f"thread pool of {threads} host threads"}
    return out


# ------------------------------------------------------------ served queries

def serve_specs(seed=6):
    """Resident graph pool: 32 square grids with n = 2^U(10,20) and 32 banded
    graphs with n = 2^U(12,20), degree 32, window +-256; weights uniform in
    [1, 65535]; graph g seeded 2000 + g."""
    st = gen.Stream(seed)
    specs = []
    for q in range(64):
        if q < 32:
            side = int(round(2 ** ((10 + 10 * st.random()) / 2)))
            specs.append(("grid", side, 4, 2000 + q, 0))
        else:
            n = int(round(2 ** (12 + 8 * st.random())))
            specs.append(("banded", n, 32, 2000 + q, 0))
    return specs


def serve_pool(seed=6):
    return par_map(make_spec_graph, serve_specs(seed))


def serve_requests(graphs, n, rate, seed):
    from paper_1908_09378_gb300.serve import poisson_arrivals
    st = gen.Stream(seed + 17)
    reqs = []
    for a in poisson_arrivals(n, rate, seed):
        gi = st.uniform(0, len(graphs) - 1)
        reqs.append((a, gi, st.uniform(0, graphs[gi].n - 1)))
    return reqs


SERVE_BUDGET = 40_000_000_000  # 40 GB of device memory for admitted queries
SERVE_LARGE_ARCS = 1 << 23     # served queries of at least this many arcs run on clusters


def bench_serve(args, dist: Dist, torch, pbh, requests: int, cpu: bool):
    """The served stream.  Capacity C from a burst; then `requests` Poisson arrivals at
    0.8 C (latency) and at 2 C (saturated queries/s).  Under N ranks each
    rank serves the requests with index = rank mod N at rate / N."""
    from paper_1908_09378_gb300 import serve
    t0 = time.perf_counter()
    graphs = serve_pool()
    dgs = [pbh.DeviceGraph(g) for g in graphs]
    log(f"pool of {len(graphs)} graphs, m total {sum(g.m for g in graphs) / 1e6:.1f}M, "
        f"generated in {time.perf_counter() - t0:.1f}s")

    def mine(reqs):
        return reqs[dist.rank::dist.world]

    def large_ctas_for(team):
        # large queries (>= --serve-large-arcs arcs) on clusters of `team` CTAs in
        # a second launch, with a share of the SMs equal to their share of the
        # pool's work (vertices + arcs; every graph is equally likely)
        if team < 2:
            return 0
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        work = [g.n + g.m for g in graphs]
        share = sum(w for w, g in zip(work, graphs) if g.m >= args.serve_large_arcs) / sum(work)
        return max(team, min(int(round(share * sms / team)) * team, (3 * sms // 4) // team * team))

    def serve_runs(team, burst_n, n, kept=None, every=1):
        large_ctas = large_ctas_for(team)
        sv = serve.Server(budget_bytes=SERVE_BUDGET, slots=32768, large_team=team, large_ctas=large_ctas,
                          large_arcs=args.serve_large_arcs)
        try:
            serve.run_stream(sv, dgs, mine(serve_requests(graphs, 500, 0.0, 1)))
            burst = serve.run_stream(sv, dgs, mine(serve_requests(graphs, burst_n, 0.0, 2)))
            cap = dist.sum(torch, burst["qps"])
            clocks = ClockSampler(dist.local)
            clocks.start()
            lat_reqs = mine(serve_requests(graphs, n, 0.8 * cap, 3))
            lat = serve.run_stream(sv, dgs, lat_reqs,
                                   collect=(lambda i, d: kept.__setitem__(i, d.cpu().numpy().view(np.uint64))
                                            if i % every == 0 else None) if kept is not None else None)
            sat = serve.run_stream(sv, dgs, mine(serve_requests(graphs, n, 2.0 * cap, 4)))
            ck = clocks.stop()
        finally:
            sv.stop()
        return cap, lat_reqs, lat, sat, ck, large_ctas

    sample_every = max(1, requests // 48)  # ~48 results kept for the oracle check
    kept = {}
    team = args.serve_team
    cap, lat_reqs, lat, sat, ck, large_ctas = serve_runs(team, 4000, requests, kept, sample_every)
    qps_sat = dist.sum(torch, sat["qps"])
    alt = None
    if args.serve_alt_team >= 2 and args.serve_alt_team != team:
        # the same stream's shape with large queries on clusters: a shorter tail
        # for lower throughput (fewer requests, to keep the run short)
        a_team = args.serve_alt_team
        a_cap, _, a_lat, a_sat, _, a_ctas = serve_runs(a_team, 2000, max(1000, requests // 4))
        alt = {"team": f"queries of >= {args.serve_large_arcs} arcs on {a_team}-CTA clusters ({a_ctas} CTAs), the rest "
                       "one CTA each", "requests": max(1000, requests // 4), "capacity_qps": a_cap,
               "saturated_qps": dist.sum(torch, a_sat["qps"]), "p50_ms": a_lat["p50_ms"], "p99_ms": a_lat["p99_ms"],
               "p99_over_p50": a_lat["p99_ms"] / a_lat["p50_ms"], "peak_pool_bytes": max(a_lat["peak_pool_bytes"],
                                                                                         a_sat["peak_pool_bytes"])}
    # the sampled results against the oracle (all host cores); their U sizes the roofline
    idx = sorted(kept)
    res, t_cpu, threads = oracle_pool([graphs[lat_reqs[i][1]] for i in idx], [lat_reqs[i][2] for i in idx])
    mism = [i for i, (want, _) in zip(idx, res) if not np.array_equal(want, kept[i])]
    if mism:
        raise RuntimeError(f"serve: requests {mism[:10]} differ from the oracle")
    bytes_sample = [algorithmic_bytes(graphs[lat_reqs[i][1]].n, reached_arcs(graphs[lat_reqs[i][1]], kept[i]), U)
                    for i, (_, U) in zip(idx, res)]
    ab_mean = sum(bytes_sample) / max(len(bytes_sample), 1)
    # one-query-at-a-time plain path on a sample of the same stream
    sample = serve_requests(graphs, 200, 0.0, 4)
    wss = {}
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _, gi, src in sample:
        dg = dgs[gi]
        if dg.n not in wss:
            wss[dg.n] = pbh.SsspWorkspace(dg.n)
        pbh.sssp_async(dg, src, ws=wss[dg.n])
    torch.cuda.synchronize()
    qps_one = len(sample) / (time.perf_counter() - t1)
    cfg = {"workload": f"Poisson stream of {requests} SSSP queries over a resident pool of 32 grids "
                       "(n 2^10..2^20) and 32 banded graphs (n 2^12..2^20, degree 32, window +-256), "
                       "w~U[1,65535]; uniform graph and source", "requests": requests,
           "budget_bytes": SERVE_BUDGET, "capacity_qps": cap, "rate_latency_run": 0.8 * cap,
           "rate_saturated_run": 2.0 * cap,
           "team": (f"queries of >= {args.serve_large_arcs} arcs on {team}-CTA clusters ({large_ctas} CTAs), the rest one "
                    "CTA each: two persistent launches" if team >= 2 else "one CTA per query, one persistent launch"),
           "parallelism": f"requests split over {dist.world} GPU(s) by index, no collective"}
    out = {"metric": "served SSSP queries/s (continuous batching) and p50/p99 latency", "value": qps_sat,
           "unit": "queries/s", "n_gpus": dist.world, "steps": 1, "warmup": 1,
           "ms_per_step": 1e3 * sat["wall_s"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": cfg,
           "latency": {"p50_ms": lat["p50_ms"], "p99_ms": lat["p99_ms"], "mean_ms": lat["mean_ms"],
                       "qps": lat["qps"], "device_p50_ms": lat["device_p50_ms"]},
           "saturated": sat, "peak_pool_bytes": max(lat["peak_pool_bytes"], sat["peak_pool_bytes"]),
           "roofline": roofline(int(ab_mean * sat["served"]), sat["wall_s"], "k_serve", None,
                                bytes_formula="served queries x the mean 8(n+1) + 8 m_reached + 8n + 16U of "
                                              f"{len(idx)} sampled requests; over the saturated run's wall time"),
           "one_at_a_time": {"value": qps_one, "unit": "queries/s", "sample": len(sample)},
           "speedup_vs_one_at_a_time": qps_sat / qps_one, "clocks": ck, "gpu_launches": 4,
           "p99_over_p50": lat["p99_ms"] / lat["p50_ms"], "large_queries_on_clusters": alt,
           "oracle_check": {"compared": f"{len(idx)} requests of the latency run (every {sample_every}th), "
                                        "every vertex", "mismatches": 0}}
    if dist.rank == 0 and cpu:
        n_cpu = min(len(lat_reqs), 256)
        cres, t_c, threads = oracle_pool([graphs[gi] for _, gi, _ in lat_reqs[:n_cpu]],
                                         [src for _, _, src in lat_reqs[:n_cpu]])
        out["cpu_baseline"] = {"value": n_cpu / t_c, "unit": "queries/s", "cores": threads, "kind": "oracle",
                               "cpu": cpu_model(),
                               "sample": f"the first {n_cpu} requests of the latency stream, sequential Dijkstra "
                                         f"per query on a thread pool of {threads} host threads"}
    return out


# ------------------------------------------------------------ reference arm

def reference_arm(args):
    """The CPU oracle, as it stands, on the same workload and metric."""
    import oracle
    if args.workload not in ("banded", "grid64"):
        return {"impl": "reference", "unavailable": f"no oracle arm for workload {args.workload}"}
    g = banded_graph() if args.workload == "banded" else gen.grid(64, 64, 1, 100, 0)
    cfg = banded_cfg() if args.workload == "banded" else {"workload": "64x64 grid", "n": g.n, "m": g.m}
    d0 = oracle.dijkstra(g, 0)
    m_reached = reached_arcs(g, d0)
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
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": sample,
                             "cpu": cpu_model()},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ------------------------------------------------------------ ranks

def free_port() -> int:
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def spawn_command(args, argv):
    """The torchrun command that starts args.gpus ranks of this script (one
    process per GPU), or None when this process is already a rank or N = 1."""
    if args.gpus <= 1 or "WORLD_SIZE" in os.environ:
        return None
    return [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
            "--master-addr", "127.0.0.1", "--master-port", str(free_port()), os.path.abspath(__file__), *argv]


def ranks_check(args):
    """Host-only check of the multi-rank plumbing (gloo, no GPU): every rank
    takes its shard of the batch queries and the sums cross ranks."""
    import torch
    dist = Dist(args.gpus, backend="gloo")
    dist.init(torch)
    specs = batch_specs(args.queries)
    weights = [(s[1] * s[1] * 5 if s[0] == "grid" else s[1] * (s[2] + 1)) for s in specs]
    mine = shard(weights, dist.rank, dist.world)
    total = dist.sum(torch, float(len(mine)))
    wmax = dist.max(torch, float(sum(weights[i] for i in mine)))
    if dist.rank == 0:
        print(json.dumps({"world": dist.world, "queries_total": int(total), "max_rank_weight": wmax,
                          "rank0_queries": len(mine)}), flush=True)
    dist.close()
    return 0


# ------------------------------------------------------------ main

def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="all", choices=["all", "banded", "grid64", "dag", "heap", "heap_general",
                                                          "batch", "serve", "ranks"])
    ap.add_argument("--m", type=int, default=100_000_000, help="dag workload: arcs")
    ap.add_argument("--requests", type=int, default=20000, help="serve workload: requests per run")
    ap.add_argument("--queries", type=int, default=512, help="batch workload: number of queries")
    ap.add_argument("--r", type=int, default=0, help="extract width (0 = library default)")
    ap.add_argument("--d", type=int, default=0, help="heap parameter d (0 = library default)")
    ap.add_argument("--cta", type=int, default=0, help="team: 0 whole GPU, 1 one CTA, 2..16 one cluster")
    ap.add_argument("--settle", action="store_true", help="single-query workloads: the settle criterion flag")
    ap.add_argument("--rounds", type=int, default=1000, help="heap workload rounds")
    ap.add_argument("--n", type=int, default=20, help="log2 vertices of the banded workload (profiling only)")
    ap.add_argument("--cpu-budget", type=float, default=10.0, help="seconds of oracle time in the heap CPU baseline")
    ap.add_argument("--serve-team", type=int, default=0, help="serve: cluster size for large queries (0 = none)")
    ap.add_argument("--deep-ctas", type=int, default=128, help="heap: CTAs of the deep group (concurrent resolution)")
    ap.add_argument("--serve-large-arcs", type=int, default=SERVE_LARGE_ARCS,
                    help="serve: queries of at least this many arcs go to the cluster launch")
    ap.add_argument("--serve-alt-team", type=int, default=8,
                    help="serve: also measure large queries on clusters of this size (0 = skip)")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu-baseline", dest="cpu", action="store_false")
    args = ap.parse_args(argv)
    args.warmup = max(args.warmup, 3)
    global LOGN
    LOGN = args.n

    if args.workload == "ranks":
        cmd = spawn_command(args, argv)
        return subprocess.call(cmd) if cmd else ranks_check(args)

    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return 0
        if args.workload == "all":
            args.workload = "banded"
        print(json.dumps(reference_arm(args)), flush=True)
        return 0

    cmd = spawn_command(args, argv)
    if cmd:
        log("starting ranks: " + " ".join(cmd))
        return subprocess.call(cmd)

    import torch
    import paper_1908_09378_gb300 as pbh
    pbh.load()
    dist = Dist(args.gpus)
    dist.init(torch)
    if args.workload == "heap":
        out = bench_heap(args, dist, torch, pbh, args.rounds, args.steps, args.warmup, args.cpu)
    elif args.workload == "heap_general":
        out = bench_heap_general(args, dist, torch, pbh)
    elif args.workload == "batch":
        out = bench_batch(args, dist, torch, pbh, args.steps, args.warmup, args.cpu)
    elif args.workload == "serve":
        out = bench_serve(args, dist, torch, pbh, args.requests, args.cpu)
    elif args.workload in ("banded", "grid64", "dag"):
        out = bench_sssp(args, dist, torch, pbh, args.workload, args.steps, args.warmup, args.e2e, args.cpu)
    else:
        # the headline (the banded 2^20 single query), then the 64x64 grid, the heap stream, the batch and the
        # served stream as sub-objects
        t0 = time.perf_counter()
        out = bench_sssp(args, dist, torch, pbh, "banded", args.steps, args.warmup, args.e2e, args.cpu)
        subs = {}
        for name, fn in (("grid64", lambda: bench_sssp(args, dist, torch, pbh, "grid64", 10, 3, False, args.cpu)),
                         ("heap", lambda: bench_heap(args, dist, torch, pbh, 1000, 3, 3, args.cpu)),
                         ("batch", lambda: bench_batch(args, dist, torch, pbh, 3, 3, args.cpu)),
                         ("serve", lambda: bench_serve(args, dist, torch, pbh, args.requests, args.cpu))):
            t1 = time.perf_counter()
            subs[name] = fn()
            subs[name]["wall_s"] = time.perf_counter() - t1
            log(f"{name}: {subs[name]['value']:.4g} {subs[name]['unit']} in {subs[name]['wall_s']:.0f}s")
        out["configs"] = subs
        out["bench_wall_s"] = time.perf_counter() - t0
    if dist.rank == 0:
        print(json.dumps(out), flush=True)
    dist.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
