"""Plain CPU oracle for the parity tests -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it, and it
shares no code with the CUDA library.

What it computes (oracle.c has the details and the citations):

* ``dijkstra``: exact single-source shortest-path distances (uint64,
  UINT64_MAX = unreachable) by sequential Dijkstra over a binary heap
  (Section 1, and the per-round semantics of parDijkstra in Section 4.1).
* ``dijkstra_counts``: the same run's counters, among them the successful
  relaxations U (arcs that lowered a tentative distance), which fix the
  heap traffic of the benchmark's roofline.
* ``bellman_ford``: the same distances by repeated relaxation sweeps
  (Section 1); pins ``dijkstra`` on tiny graphs.
* ``check_sssp``: the optimality certificate of a distance vector.
* ``hop_depth``: fewest arcs on a shortest path, maximised over vertices.
* ``SortedPQ``: the priority-queue ADT of Section 1.2 (BulkUpdate with
  decrease-only min semantics, extractMin of the r smallest in ascending
  (priority, key) order) as a plain sorted array.

Every function is pinned by ``tests/test_oracle.py`` against brute force,
closed forms and invariants; nothing here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lib = None

INF = np.uint64(0xFFFFFFFFFFFFFFFF)


def build(force: bool = False) -> str:
    """Compile oracle.c into _liboracle.so next to it (atomic rename)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    subprocess.run(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC],
                   check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    u32, u64, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
    for name, res, args in [
        ("oracle_dijkstra", u64, [u32, vp, vp, vp, u32, vp, vp]),
        ("oracle_dijkstra_counts", u64, [u32, vp, vp, vp, u32, vp, vp]),
        ("oracle_bellman_ford", u64, [u32, vp, vp, vp, u32, vp]),
        ("oracle_check_sssp", u64, [u32, vp, vp, vp, u32, vp, vp]),
        ("oracle_hop_depth", u32, [u32, vp, vp, vp, u32, vp, vp]),
        ("oracle_reached_edges", u64, [u32, vp, vp]),
        ("opq_create", vp, [u32]),
        ("opq_destroy", None, [vp]),
        ("opq_size", u64, [vp]),
        ("opq_bulk_update", u64, [vp, vp, vp, u32]),
        ("opq_extract_min", u32, [vp, u32, vp, vp]),
        ("opq_priority", u64, [vp, u32]),
        ("opq_assign", u64, [vp, vp, vp, u32]),
        ("opq_delete", u64, [vp, vp, u32]),
    ]:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _p(a):
    return None if a is None else a.ctypes.data


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.uint64)
    col = np.ascontiguousarray(g.col, dtype=np.uint32)
    w = np.ascontiguousarray(g.w, dtype=np.uint32)
    return rp, col, w


def dijkstra(g, source: int, want_parent: bool = False):
    """Exact distances from source (uint64; INF = unreachable)."""
    lib = _load()
    rp, col, w = _csr(g)
    dist = np.empty(g.n, dtype=np.uint64)
    parent = np.empty(g.n, dtype=np.uint32) if want_parent else None
    lib.oracle_dijkstra(g.n, _p(rp), _p(col), _p(w), source, _p(dist), _p(parent))
    return (dist, parent) if want_parent else dist


def dijkstra_counts(g, source: int):
    """(dist, settled, scanned arcs, successful relaxations U) of one Dijkstra run."""
    lib = _load()
    rp, col, w = _csr(g)
    dist = np.empty(g.n, dtype=np.uint64)
    counts = np.zeros(3, dtype=np.uint64)
    lib.oracle_dijkstra_counts(g.n, _p(rp), _p(col), _p(w), source, _p(dist), _p(counts))
    return dist, int(counts[0]), int(counts[1]), int(counts[2])


def bellman_ford(g, source: int):
    lib = _load()
    rp, col, w = _csr(g)
    dist = np.empty(g.n, dtype=np.uint64)
    lib.oracle_bellman_ford(g.n, _p(rp), _p(col), _p(w), source, _p(dist))
    return dist


def check_sssp(g, source: int, dist) -> np.ndarray:
    """Violation counts [dist[s]!=0, arc violations, untight reached, reachability]."""
    lib = _load()
    rp, col, w = _csr(g)
    d = np.ascontiguousarray(dist, dtype=np.uint64)
    counts = np.zeros(4, dtype=np.uint64)
    lib.oracle_check_sssp(g.n, _p(rp), _p(col), _p(w), source, _p(d), _p(counts))
    return counts


def hop_depth(g, source: int, dist, want_hops: bool = False):
    lib = _load()
    rp, col, w = _csr(g)
    d = np.ascontiguousarray(dist, dtype=np.uint64)
    hops = np.empty(g.n, dtype=np.uint32) if want_hops else None
    H = int(lib.oracle_hop_depth(g.n, _p(rp), _p(col), _p(w), source, _p(d), _p(hops)))
    return (H, hops) if want_hops else H


def reached_edges(g, dist) -> int:
    lib = _load()
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.uint64)
    d = np.ascontiguousarray(dist, dtype=np.uint64)
    return int(lib.oracle_reached_edges(g.n, _p(rp), _p(d)))


class SortedPQ:
    """Sorted-array priority queue (the ADT of Section 1.2)."""

    def __init__(self, key_space: int):
        lib = _load()
        self.key_space = key_space
        self._q = lib.opq_create(key_space)

    def bulk_update(self, keys, prios) -> int:
        k = np.ascontiguousarray(keys, dtype=np.uint32)
        p = np.ascontiguousarray(prios, dtype=np.uint32)
        assert len(k) == len(p)
        return int(_lib.opq_bulk_update(self._q, _p(k), _p(p), len(k)))

    def assign(self, keys, prios) -> int:
        """update with replace semantics (Section 1.2, footnote): the last
        element of each key in the batch wins, up or down."""
        k = np.ascontiguousarray(keys, dtype=np.uint32)
        p = np.ascontiguousarray(prios, dtype=np.uint32)
        assert len(k) == len(p)
        return int(_lib.opq_assign(self._q, _p(k), _p(p), len(k)))

    def delete(self, keys) -> int:
        """delete (Section 1.2) of every listed key that is live."""
        k = np.ascontiguousarray(keys, dtype=np.uint32)
        return int(_lib.opq_delete(self._q, _p(k), len(k)))

    def extract_min(self, r: int):
        keys = np.empty(max(r, 1), dtype=np.uint32)
        prios = np.empty(max(r, 1), dtype=np.uint32)
        c = int(_lib.opq_extract_min(self._q, r, _p(keys), _p(prios)))
        return keys[:c].copy(), prios[:c].copy()

    def priority(self, key: int) -> int:
        return int(_lib.opq_priority(self._q, key))

    def __len__(self):
        return int(_lib.opq_size(self._q))

    def __del__(self):
        if getattr(self, "_q", None) and _lib is not None:
            _lib.opq_destroy(self._q)
            self._q = None
