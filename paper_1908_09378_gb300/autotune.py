"""Parameter choice for batched and single queries: the extract width r, the
heap parameter d (the level capacities: bucket B_i holds 2 d 4^i words) and
the team (one CTA, a thread-block cluster of 2-16 CTAs, or the whole GPU).

Batched queries are grouped into size classes by (log2 n, out-degree
bucket).  For each class the table holds the (r, d multiplier) that measured
fastest on this GPU for a one-CTA team; d is the smallest power of two >=
r * max_degree, times the multiplier, so a round's BulkUpdate always fits
(Section 4.1 sets d to the maximum degree for r = 1).  On top of that, the
largest queries of a batch run on thread-block clusters: the cluster size and
the arc count from which a query gets one are searched on the batch itself
(`tune_batch_teams`), since a one-CTA query of many arcs sets the batch's
makespan.  Single queries have their own table of (team, r, d) per class.
`tune()` / `tune_single()` measure on sample queries and write a JSON cache
keyed by GPU name; without a cache entry the built-in defaults below are used.
"""
from __future__ import annotations

import json
import math
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.environ.get("PBH_TUNE_CACHE", os.path.join(HERE, "tuned.json"))
CANDIDATES = (16, 32, 64, 128, 256, 512, 1024)
D_MULTIPLIERS = (1, 2, 4)
TEAM_CANDIDATES = ((0, 0), (2, 1 << 23), (4, 1 << 22), (4, 1 << 23), (4, 1 << 24), (8, 1 << 22), (8, 1 << 23),
                   (8, 1 << 24), (16, 1 << 23))
SINGLE_TEAMS = (1, 4, 8, 16, 0)
SINGLE_R = (64, 128, 256, 384, 512, 768, 1024, 1536, 2048)
SINGLE_D = (1 << 15, 1 << 16, 1 << 17, 1 << 18, 1 << 19, 1 << 20, 1 << 21)

# r by size class for one-CTA teams, before tuning: grows with n so that
# rounds stay near the hop depth without flooding one CTA with arcs
DEFAULT_R = {10: 16, 11: 16, 12: 16, 13: 32, 14: 32, 15: 64, 16: 64, 17: 128, 18: 128, 19: 256, 20: 256}

_table = None
_source = "defaults"


def size_class(n: int, max_degree: int) -> str:
    lg = max(10, min(20, int(round(math.log2(max(n, 2))))))
    db = "lo" if max_degree <= 8 else "hi"
    return f"{lg}{db}"


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "unknown"


def _load():
    global _table, _source
    if _table is not None:
        return _table
    _table = {}
    if os.path.exists(CACHE):
        try:
            with open(CACHE) as f:
                allt = json.load(f)
            _table = allt.get(_gpu_name(), {})
            if _table:
                _source = f"tuned ({os.path.basename(CACHE)})"
        except (OSError, ValueError):
            _table = {}
    return _table


def _entry(c):
    """(r, d multiplier) of a batch size class (older caches hold r alone)."""
    v = _load().get(c)
    if v is None:
        return None
    if isinstance(v, dict):
        return int(v["r"]), int(v.get("dmul", 1))
    return int(v), 1


def r_for(n: int, max_degree: int) -> int:
    e = _entry(size_class(n, max_degree))
    if e:
        return e[0]
    lg = max(10, min(20, int(round(math.log2(max(n, 2))))))
    return DEFAULT_R[lg]


def d_for(r: int, max_degree: int, mul: int = 1) -> int:
    need = max(1, r * max(max_degree, 1))
    return (1 << (need - 1).bit_length()) * mul


def teams() -> tuple:
    """(cluster size, arc threshold) for the large queries of a batch; (0, 0)
    keeps every query on one CTA."""
    t = _load().get("batch_teams")
    if t:
        return int(t[0]), int(t[1])
    return 8, 1 << 22


def batch_params(dgs, team=None):
    """Per query: r, d and the team (1 = one CTA, k >= 2 = a cluster of k)."""
    k, thr = teams() if team is None else team
    rs, ds, cs = [], [], []
    for g in dgs:
        e = _entry(size_class(g.n, g.max_degree))
        r, mul = e if e else (r_for(g.n, g.max_degree), 1)
        rs.append(r)
        ds.append(d_for(r, g.max_degree, mul))
        cs.append(k if k >= 2 and g.m >= thr else 1)
    return rs, ds, cs


def single_params(n: int, m: int, max_degree: int):
    """(cta, r, d) for one query on its own: the tuned entry of its class, else
    the library's choice (cta 16 up to 2^19 arcs, else the whole GPU)."""
    v = _load().get("single", {}).get(size_class(n, max_degree))
    if v:
        return int(v["cta"]), int(v["r"]), int(v["d"])
    return (16 if m <= (1 << 19) else 0), 512, 1 << 16


def team_params(n: int, max_degree: int, team: int):
    """(r, d) for one query on a given team (0 = whole GPU, k = a k-CTA
    cluster, 1 = one CTA): the single-query tuner's best on that team for
    the query's class, else the batch rule's (one-CTA) r and d."""
    v = _load().get("single_teams", {}).get(size_class(n, max_degree), {}).get(str(team))
    if v and team != 1:
        return int(v["r"]), int(v["d"])
    e = _entry(size_class(n, max_degree))
    r, mul = e if e else (r_for(n, max_degree), 1)
    return r, d_for(r, max_degree, mul)


def describe_single(n: int, max_degree: int) -> str:
    c = size_class(n, max_degree)
    if _load().get("single", {}).get(c):
        return f"size class {c} of the single-query table ({_source})"
    return f"size class {c}: the library's choice (no tuned entry)"


def describe() -> str:
    _load()
    k, thr = teams()
    return (f"r and d per size class from {_source}; d = next power of two >= r * max degree, times the "
            f"class's multiplier; queries of >= {thr} arcs on {k}-CTA clusters" if k else
            f"r and d per size class from {_source}; every query on one CTA")


def _time(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        fn()
        e.record()
        torch.cuda.synchronize()
        ts.append(s.elapsed_time(e))
    return min(ts)


def _write(update: dict):
    allt = {}
    if os.path.exists(CACHE):
        try:
            with open(CACHE) as f:
                allt = json.load(f)
        except (OSError, ValueError):
            allt = {}
    allt.setdefault(_gpu_name(), {}).update(update)
    tmp = CACHE + f".tmp{os.getpid()}.{int(time.time())}"
    with open(tmp, "w") as f:
        json.dump(allt, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)
    global _table
    _table = None


def tune(graphs_by_class, sources_by_class, reps: int = 2, write: bool = True):
    """Measure each candidate (r, d multiplier) on each class's sample (run as
    one batch, one CTA per query) and keep the fastest.  Returns
    {class: {"r": r, "dmul": mul, "ms": time}} plus the timing grid."""
    import paper_1908_09378_gb300 as pbh
    best, grid = {}, {}
    for c, dgs in graphs_by_class.items():
        srcs = sources_by_class[c]
        timing = {}
        for r in CANDIDATES:
            for mul in D_MULTIPLIERS:
                ds = [d_for(r, g.max_degree, mul) for g in dgs]
                b = pbh.Batch(dgs, srcs, r=[r] * len(dgs), d=ds, cta=1)
                timing[(r, mul)] = _time(lambda: (b.run_async(), b.status()), reps)
        (r, mul) = min(timing, key=timing.get)
        best[c] = {"r": r, "dmul": mul, "ms": round(timing[(r, mul)], 3)}
        grid[c] = {f"r{r}_d{m}": round(v, 3) for (r, m), v in timing.items()}
    if write:
        _write(best)
    return best, grid


def tune_batch_teams(dgs, sources, reps: int = 2, write: bool = True):
    """The batch's team rule: for each (cluster size, arc threshold) candidate
    run the whole batch and keep the fastest.  Returns (best, {candidate: ms})."""
    import paper_1908_09378_gb300 as pbh
    timing = {}
    for k, thr in TEAM_CANDIDATES:
        rs, ds, cs = batch_params(dgs, team=(k, thr))
        b = pbh.Batch(dgs, sources, r=rs, d=ds, cta=cs)
        timing[(k, thr)] = _time(lambda: (b.run_async(), b.status()), reps)
    best = min(timing, key=timing.get)
    if write:
        _write({"batch_teams": [int(best[0]), int(best[1])]})
    return best, {f"k{k}_m{thr}": round(v, 3) for (k, thr), v in timing.items()}


def tune_single(graphs_by_class, reps: int = 2, write: bool = True):
    """One query per class sample (source 0) on each team, r and d; keeps the
    fastest, and the fastest (r, d) of every team (for callers that fix the
    team, such as the server's cluster launch).  Returns ({class: {"cta",
    "r", "d", "ms"}}, timing grid, {class: {team: {"r", "d", "ms"}}})."""
    import paper_1908_09378_gb300 as pbh
    best, grid, by_team = {}, {}, {}
    for c, g in graphs_by_class.items():
        timing = {}
        for cta in SINGLE_TEAMS:
            if cta == 1 and g.n >= (1 << 16):
                continue  # one CTA never wins from 2^16 vertices on (seconds per candidate)
            for r in SINGLE_R:
                for d in SINGLE_D:
                    if r * max(g.max_degree, 1) > d:
                        continue
                    ws = pbh.SsspWorkspace(g.n, r, d, cta)
                    dist = pbh._torch().empty(max(g.n, 1), dtype=pbh._torch().int64, device="cuda")
                    try:
                        timing[(cta, r, d)] = _time(lambda: pbh.sssp_async(g, 0, dist=dist, ws=ws), reps)
                        pbh.sssp_stats(ws)  # a latched device error disqualifies the candidate
                    except pbh.PbhError:
                        timing.pop((cta, r, d), None)
                        continue
        key = min(timing, key=timing.get)
        best[c] = {"cta": key[0], "r": key[1], "d": key[2], "ms": round(timing[key], 4)}
        grid[c] = {f"t{a}_r{b}_d{d}": round(v, 4) for (a, b, d), v in timing.items()}
        by_team[c] = {}
        for (a, b, d), v in sorted(timing.items(), key=lambda kv: kv[1]):
            by_team[c].setdefault(str(a), {"r": b, "d": d, "ms": round(v, 4)})
    if write:
        _write({"single": best, "single_teams": by_team})
    return best, grid, by_team


def sample_classes(per_class: int = 8, seed: int = 31):
    """Sample queries for every size class: square grids (low degree) and
    banded graphs (degree 32, window +-256) with n near 2^lg."""
    import gen
    st = gen.Stream(seed)
    graphs, sources = {}, {}
    for lg in range(10, 21, 2):
        for kind in ("lo", "hi"):
            gs, ss = [], []
            for q in range(per_class):
                if kind == "lo":
                    side = int(round(2 ** (lg / 2)))
                    g = gen.grid(side, side, 1, 65535, 7000 + 97 * lg + q)
                else:
                    g = gen.banded(1 << lg, 32, 256, 1, 65535, 8000 + 97 * lg + q)
                gs.append(g)
                ss.append(st.uniform(0, g.n - 1))
            graphs[f"{lg}{kind}"] = gs
            sources[f"{lg}{kind}"] = ss
    return graphs, sources


def single_classes(seed: int = 41):
    """One sample graph per single-query class: square grids and banded graphs
    (degree 64, window +-512) with n near 2^lg."""
    import gen
    out = {}
    for lg in range(12, 21, 2):
        side = int(round(2 ** (lg / 2)))
        out[f"{lg}lo"] = gen.grid(side, side, 1, 65535, seed + lg)
        out[f"{lg}hi"] = gen.banded(1 << lg, 64, 512, 1, 65535, seed + 100 + lg)
    return out


if __name__ == "__main__":
    import sys
    import paper_1908_09378_gb300 as pbh
    pbh.load()
    what = sys.argv[1] if len(sys.argv) > 1 else "batch"
    if what == "batch":
        gs, ss = sample_classes(int(sys.argv[2]) if len(sys.argv) > 2 else 8)
        dgs = {c: [pbh.DeviceGraph(g) for g in v] for c, v in gs.items()}
        best, grid = tune(dgs, ss, write=False)
        # odd sizes take the entry of the even class below them
        for c, v in list(best.items()):
            lg, kind = int(c[:-2]), c[-2:]
            best.setdefault(f"{lg + 1}{kind}", v)
        _write(best)
        print(json.dumps({"best": best, "grid": grid}, sort_keys=True))
    elif what == "teams":
        import bench
        graphs, sources = bench.batch_queries()
        dgs = [pbh.DeviceGraph(g) for g in graphs]
        best, grid = tune_batch_teams(dgs, sources)
        print(json.dumps({"best": list(best), "grid": grid}, sort_keys=True))
    elif what == "single":
        gs = single_classes()
        dgs = {c: pbh.DeviceGraph(g) for c, g in gs.items()}
        best, grid, by_team = tune_single(dgs, write=False)
        for c in list(best):
            lg, kind = int(c[:-2]), c[-2:]
            best.setdefault(f"{lg + 1}{kind}", best[c])
            by_team.setdefault(f"{lg + 1}{kind}", by_team[c])
        _write({"single": best, "single_teams": by_team})
        print(json.dumps({"best": best, "grid": grid}, sort_keys=True))
