"""Parameter choice for batched queries (extract width r and heap parameter d
per query).

Queries are grouped into size classes by (log2 n, out-degree bucket).  For
each class the table holds the r that measured fastest on this GPU for a
one-CTA team; d is then the smallest power of two >= r * max_degree, so a
round's BulkUpdate always fits (Section 4.1 sets d to the maximum degree for
r = 1).  `tune()` measures the table on sample queries and writes it to a
JSON cache keyed by GPU name; without a cache entry the built-in defaults
below are used.
"""
from __future__ import annotations

import json
import math
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.environ.get("PBH_TUNE_CACHE", os.path.join(HERE, "tuned.json"))
CANDIDATES = (16, 32, 64, 128, 256)

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


def r_for(n: int, max_degree: int) -> int:
    t = _load()
    c = size_class(n, max_degree)
    if c in t:
        return int(t[c])
    lg = max(10, min(20, int(round(math.log2(max(n, 2))))))
    return DEFAULT_R[lg]


def d_for(r: int, max_degree: int) -> int:
    need = max(1, r * max(max_degree, 1))
    return 1 << (need - 1).bit_length()


def batch_params(dgs):
    rs, ds = [], []
    for g in dgs:
        r = r_for(g.n, g.max_degree)
        rs.append(r)
        ds.append(d_for(r, g.max_degree))
    return rs, ds


def describe() -> str:
    _load()
    return f"r per size class from {_source}; d = next power of two >= r * max degree"


def tune(graphs_by_class, sources_by_class, reps: int = 2, write: bool = True):
    """Measure each candidate r on each class's sample (run as one batch, one
    CTA per query) and keep the fastest.  Returns {class: r}."""
    import torch
    import paper_1908_09378_gb300 as pbh
    best = {}
    for c, dgs in graphs_by_class.items():
        srcs = sources_by_class[c]
        timing = {}
        for r in CANDIDATES:
            ds = [d_for(r, g.max_degree) for g in dgs]
            b = pbh.Batch(dgs, srcs, r=[r] * len(dgs), d=ds)
            b.run_async()
            b.status()
            ts = []
            for _ in range(reps):
                s = torch.cuda.Event(enable_timing=True)
                e = torch.cuda.Event(enable_timing=True)
                s.record()
                b.run_async()
                e.record()
                torch.cuda.synchronize()
                ts.append(s.elapsed_time(e))
            timing[r] = min(ts)
        best[c] = min(timing, key=timing.get)
    if write:
        allt = {}
        if os.path.exists(CACHE):
            try:
                with open(CACHE) as f:
                    allt = json.load(f)
            except (OSError, ValueError):
                allt = {}
        allt.setdefault(_gpu_name(), {}).update({k: int(v) for k, v in best.items()})
        tmp = CACHE + f".tmp{os.getpid()}.{int(time.time())}"
        with open(tmp, "w") as f:
            json.dump(allt, f, indent=1, sort_keys=True)
        os.replace(tmp, CACHE)
        global _table
        _table = None
    return best


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


if __name__ == "__main__":
    import sys
    import paper_1908_09378_gb300 as pbh
    pbh.load()
    gs, ss = sample_classes(int(sys.argv[1]) if len(sys.argv) > 1 else 8)
    dgs = {c: [pbh.DeviceGraph(g) for g in v] for c, v in gs.items()}
    best = tune(dgs, ss, write=False)
    # odd sizes take the r of the even class below them
    for c, r in list(best.items()):
        lg, kind = int(c[:-2]), c[-2:]
        best.setdefault(f"{lg + 1}{kind}", r)
    allt = {}
    if os.path.exists(CACHE):
        with open(CACHE) as f:
            allt = json.load(f)
    allt.setdefault(_gpu_name(), {}).update({k: int(v) for k, v in best.items()})
    with open(CACHE, "w") as f:
        json.dump(allt, f, indent=1, sort_keys=True)
    print(json.dumps(best, sort_keys=True))
