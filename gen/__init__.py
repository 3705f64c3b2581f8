"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module draws graphs and heap update batches; it holds no shortest-path or
priority-queue arithmetic.  The C source (gen.c) is compiled with the host C
compiler on first use; everything is deterministic for a fixed seed on any
machine (SplitMix64 stream, exact rejection sampling).

Workload recipes (shapes follow the paper's regime of large, dense, high
diameter graphs, Section 4.2, and the five configurations this library is
measured on):

* grid(rows, cols, wlo, whi, seed): 4-neighbour directed grid, row-major ids.
* banded(n, deg, win, wlo, whi, seed): vertex i -> deg distinct targets drawn
  uniformly from [i-win, i+win] clipped to [0, n-1], excluding i.
* dag(n, m, seed): the paper's random DAG (chain of weight-1 arcs plus extra
  forward arcs (u, v) of weight 2(v-u)), 0-indexed.
* random_graph(n, m, wlo, whi, seed): m uniform arcs (tests only).
* HeapStream: closed-loop update-batch generator for the heap op stream.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_libgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into _libgen.so next to it (atomic rename)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=_HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    u32, u64, vp = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
    lib.gen_grid_edges.restype = u64
    lib.gen_grid_edges.argtypes = [u32, u32]
    lib.gen_grid.restype = None
    lib.gen_grid.argtypes = [u32, u32, u32, u32, u64, vp, vp, vp]
    lib.gen_banded_edges.restype = u64
    lib.gen_banded_edges.argtypes = [u32, u32, u32]
    lib.gen_banded.restype = None
    lib.gen_banded.argtypes = [u32, u32, u32, u32, u32, u64, vp, vp, vp]
    lib.gen_random_graph.restype = None
    lib.gen_random_graph.argtypes = [u32, u64, u32, u32, u64, vp, vp, vp]
    lib.gen_dag_degrees.restype = u64
    lib.gen_dag_degrees.argtypes = [u32, u64, vp]
    lib.gen_dag.restype = None
    lib.gen_dag.argtypes = [u32, u64, u64, vp, vp, vp]
    lib.gen_uniform_array_u32.restype = None
    lib.gen_uniform_array_u32.argtypes = [u64, u32, u32, vp, u64]
    lib.gen_splitmix64.restype = u64
    lib.gen_splitmix64.argtypes = [ctypes.POINTER(u64)]
    lib.gen_uniform.restype = u64
    lib.gen_uniform.argtypes = [ctypes.POINTER(u64), u64, u64]
    lib.hs_create.restype = vp
    lib.hs_create.argtypes = [u32, u64]
    lib.hs_destroy.restype = None
    lib.hs_destroy.argtypes = [vp]
    lib.hs_nlive.restype = u32
    lib.hs_nlive.argtypes = [vp]
    lib.hs_next_batch.restype = u32
    lib.hs_next_batch.argtypes = [vp, u32, vp, vp]
    lib.hs_observe_extracted.restype = None
    lib.hs_observe_extracted.argtypes = [vp, vp, u32]
    _lib = lib
    return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Graph:
    """A CSR graph in host memory: row_ptr u64[n+1], col u32[m], w u32[m]."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def max_degree(self) -> int:
        if self.n == 0:
            return 0
        return int(np.max(np.diff(self.row_ptr))) if self.n else 0

    @property
    def nbytes(self) -> int:
        return self.row_ptr.nbytes + self.col.nbytes + self.w.nbytes


def grid(rows: int, cols: int, wlo: int = 1, whi: int = 100, seed: int = 0) -> Graph:
    lib = _load()
    n = rows * cols
    m = int(lib.gen_grid_edges(rows, cols)) if n else 0
    rp = np.zeros(n + 1, dtype=np.uint64)
    col = np.zeros(max(m, 1), dtype=np.uint32)
    w = np.zeros(max(m, 1), dtype=np.uint32)
    lib.gen_grid(rows, cols, wlo, whi, seed, _ptr(rp), _ptr(col), _ptr(w))
    return Graph(n, rp, col[:m], w[:m], f"grid{rows}x{cols}")


def banded(n: int, deg: int, win: int, wlo: int = 1, whi: int = 65535, seed: int = 1) -> Graph:
    lib = _load()
    m = int(lib.gen_banded_edges(n, deg, win))
    rp = np.zeros(n + 1, dtype=np.uint64)
    col = np.zeros(max(m, 1), dtype=np.uint32)
    w = np.zeros(max(m, 1), dtype=np.uint32)
    lib.gen_banded(n, deg, win, wlo, whi, seed, _ptr(rp), _ptr(col), _ptr(w))
    return Graph(n, rp, col[:m], w[:m], f"banded_n{n}_d{deg}_w{win}")


def random_graph(n: int, m: int, wlo: int = 1, whi: int = 100, seed: int = 0) -> Graph:
    lib = _load()
    rp = np.zeros(n + 1, dtype=np.uint64)
    col = np.zeros(max(m, 1), dtype=np.uint32)
    w = np.zeros(max(m, 1), dtype=np.uint32)
    lib.gen_random_graph(n, m, wlo, whi, seed, _ptr(rp), _ptr(col), _ptr(w))
    return Graph(n, rp, col[:m], w[:m], f"random_n{n}_m{m}")


def dag(n: int, m: int, seed: int = 0) -> Graph:
    """The paper's random DAG (Section 4.2), 0-indexed; source 0 gives dist(v) = v."""
    lib = _load()
    deg = np.zeros(max(n, 1), dtype=np.uint64)
    mm = int(lib.gen_dag_degrees(n, m, _ptr(deg)))
    rp = np.zeros(n + 1, dtype=np.uint64)
    col = np.zeros(max(mm, 1), dtype=np.uint32)
    w = np.zeros(max(mm, 1), dtype=np.uint32)
    lib.gen_dag(n, m, seed, _ptr(rp), _ptr(col), _ptr(w))
    return Graph(n, rp, col[:mm], w[:mm], f"dag_n{n}_m{mm}")


def uniform_u32(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    lib = _load()
    out = np.zeros(max(count, 1), dtype=np.uint32)
    lib.gen_uniform_array_u32(seed, lo, hi, _ptr(out), count)
    return out[:count]


class Stream:
    """A SplitMix64 stream for small seeded draws (sources, sizes, arrivals)."""

    def __init__(self, seed: int):
        self._s = ctypes.c_uint64(seed & 0xFFFFFFFFFFFFFFFF)
        _load()

    def next(self) -> int:
        return int(_lib.gen_splitmix64(ctypes.byref(self._s)))

    def uniform(self, lo: int, hi: int) -> int:
        return int(_lib.gen_uniform(ctypes.byref(self._s), lo, hi))

    def random(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next() >> 11) * (1.0 / 9007199254740992.0)


class HeapStream:
    """Closed-loop update-batch generator (see gen.c: hs_*).

    next_batch() returns (keys u32, prios u32) of distinct keys; the caller
    reports extracted keys back with observe_extracted(keys).
    """

    def __init__(self, key_space: int, seed: int = 2):
        lib = _load()
        self.key_space = key_space
        self._h = lib.hs_create(key_space, seed)

    def next_batch(self, batch: int):
        keys = np.zeros(batch, dtype=np.uint32)
        prios = np.zeros(batch, dtype=np.uint32)
        cnt = _lib.hs_next_batch(self._h, batch, _ptr(keys), _ptr(prios))
        return keys[:cnt], prios[:cnt]

    def observe_extracted(self, keys: np.ndarray) -> None:
        keys = np.ascontiguousarray(keys, dtype=np.uint32)
        _lib.hs_observe_extracted(self._h, _ptr(keys), len(keys))

    @property
    def nlive(self) -> int:
        return int(_lib.hs_nlive(self._h))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hs_destroy(self._h)
            self._h = None


def sssp_configs():
    """Named single-query workloads: the 64x64 grid (weights in [1, 100], seed 0)
    and the banded graph of 2^20 vertices (64 arcs each within +-512, weights in
    [1, 65535], seed 1), both from source 0."""
    return {
        "grid64": dict(kind="grid", rows=64, cols=64, wlo=1, whi=100, seed=0, source=0),
        "banded_n2^20": dict(kind="banded", n=1 << 20, deg=64, win=512, wlo=1, whi=65535,
                             seed=1, source=0),
    }


def make_graph(spec: dict) -> Graph:
    kind = spec["kind"]
    if kind == "grid":
        return grid(spec["rows"], spec["cols"], spec.get("wlo", 1), spec.get("whi", 100),
                    spec.get("seed", 0))
    if kind == "banded":
        return banded(spec["n"], spec["deg"], spec["win"], spec.get("wlo", 1),
                      spec.get("whi", 65535), spec.get("seed", 1))
    if kind == "dag":
        return dag(spec["n"], spec["m"], spec.get("seed", 0))
    if kind == "random":
        return random_graph(spec["n"], spec["m"], spec.get("wlo", 1), spec.get("whi", 100),
                            spec.get("seed", 0))
    raise ValueError(f"unknown graph kind {kind!r}")
