"""GB300 parallel bucket heap (parBucketHeap) and parDijkstra -- Python binding.

Argument marshalling over the C ABI of include/pbh.h (libpbh.so, built
in-tree by paper_1908_09378_gb300.build).  Every step of the computation runs
in the library's CUDA kernels; PyTorch only provides device memory and the
stream.  There is no CPU path: if the library is missing this module raises.

uint32 / uint64 data travel as int32 / int64 tensors with the same bits.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, byref, c_char_p, c_size_t, c_uint32, c_uint64, c_void_p

import numpy as np

from . import build as _build

__all__ = [
    "load", "PbhError", "Heap", "DeviceGraph", "sssp", "sssp_stats", "sssp_host", "Batch",
    "INF",
]

INF = np.uint64(0xFFFFFFFFFFFFFFFF)

STATUS = {0: "PBH_OK", 1: "PBH_E_INVAL", 2: "PBH_E_NOMEM", 3: "PBH_E_CAPACITY", 4: "PBH_E_RANGE",
          5: "PBH_E_TIMEOUT", 6: "PBH_E_CUDA"}


SSSP_SETTLE = 0x10  # sssp_opts.flags: settle criterion (extra vertices proved final each round)
SSSP_DEBUG_STALL = 0x100  # sssp_opts.flags: tests of the timeout path only (a withheld barrier arrival)


class PbhError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} {msg}".strip())


class _Params(Structure):
    _fields_ = [("key_space", c_uint32), ("d", c_uint32), ("capacity", c_uint64)]


class _Csr(Structure):
    _fields_ = [("n", c_uint32), ("m", c_uint64), ("row_ptr", c_void_p), ("col", c_void_p)]


class _Opts(Structure):
    _fields_ = [("r", c_uint32), ("d", c_uint32), ("cta", c_uint32), ("flags", c_uint32),
                ("limit_ms", c_uint32), ("wait_us", c_uint32)]


class _Stats(Structure):
    _fields_ = [("rounds", c_uint64), ("extracted", c_uint64), ("relaxations", c_uint64),
                ("improvements", c_uint64), ("stale_dropped", c_uint64), ("merged", c_uint64),
                ("resolves", c_uint64 * 16), ("t_relax_ns", c_uint64), ("t_sort_ns", c_uint64),
                ("t_empty0_ns", c_uint64), ("t_fill0_ns", c_uint64), ("t_deeper_ns", c_uint64),
                ("t_ensure_ns", c_uint64), ("barriers", c_uint64), ("levels", c_uint32), ("r_eff", c_uint32),
                ("max_degree", c_uint32), ("status", c_uint32), ("settled", c_uint64)]


class _Op(Structure):
    _fields_ = [("kind", c_uint32), ("count", c_uint32), ("r", c_uint32), ("reserved", c_uint32),
                ("d_keys", c_void_p), ("d_prios", c_void_p), ("d_keys_out", c_void_p), ("d_prios_out", c_void_p),
                ("d_count_out", c_void_p)]


OP_BULK_UPDATE, OP_EXTRACT = 0, 1


class _Query(Structure):
    _fields_ = [("g", _Csr), ("d_weights", c_void_p), ("source", c_uint32), ("d_dist_out", c_void_p),
                ("r", c_uint32), ("d", c_uint32), ("cta", c_uint32)]


_lib = None

# (name, restype, argtypes) of every symbol include/pbh.h declares
SIGNATURES = [
    ("pbh_workspace_bytes", c_size_t, [POINTER(_Params)]),
    ("pbh_create", c_uint32, [POINTER(c_void_p), POINTER(_Params), c_void_p, c_size_t, c_void_p]),
    ("pbh_bulk_update", c_uint32, [c_void_p, c_void_p, c_void_p, c_uint32]),
    ("pbh_assign", c_uint32, [c_void_p, c_void_p, c_void_p, c_uint32]),
    ("pbh_delete", c_uint32, [c_void_p, c_void_p, c_uint32]),
    ("pbh_extract_min", c_uint32, [c_void_p, c_uint32, c_void_p, c_void_p, c_void_p]),
    ("pbh_run_ops", c_uint32, [c_void_p, POINTER(_Op), c_uint32, c_uint32]),
    ("pbh_size", c_uint32, [c_void_p, POINTER(c_uint64)]),
    ("pbh_sync", c_uint32, [c_void_p]),
    ("pbh_validate", c_uint32, [c_void_p, POINTER(c_uint32), POINTER(c_uint64)]),
    ("pbh_destroy", c_uint32, [c_void_p]),
    ("sssp_workspace_bytes", c_size_t, [c_uint32, POINTER(_Opts)]),
    ("sssp_run", c_uint32, [POINTER(_Csr), c_void_p, c_uint32, c_void_p, POINTER(_Opts), c_void_p, c_size_t,
                            c_void_p]),
    ("sssp_host_workspace_bytes", c_size_t, [c_uint32, c_uint64, POINTER(_Opts)]),
    ("sssp_run_host", c_uint32, [c_uint32, c_uint64, c_void_p, c_void_p, c_void_p, c_uint32, c_void_p,
                                 POINTER(_Opts), c_void_p, c_size_t, c_void_p]),
    ("sssp_stats", c_uint32, [c_void_p, POINTER(_Stats), c_void_p]),
    ("pbh_stats", c_uint32, [c_void_p, POINTER(_Stats)]),
    ("sssp_batch_workspace_bytes", c_size_t, [POINTER(_Query), c_uint32]),
    ("sssp_batch_run", c_uint32, [POINTER(_Query), c_uint32, c_void_p, c_size_t, c_void_p]),
    ("sssp_batch_status", c_uint32, [c_void_p, c_uint32, POINTER(c_uint32), POINTER(c_uint64), c_void_p]),
    ("srv_workspace_bytes", c_size_t, []),
    ("srv_query_workspace_bytes", c_size_t, [POINTER(_Query)]),
    ("srv_create", c_uint32, [POINTER(c_void_p), c_uint32, c_uint32, c_void_p, c_size_t, c_void_p]),
    ("srv_create_team", c_uint32, [POINTER(c_void_p), c_uint32, c_uint32, c_uint32, c_void_p, c_size_t, c_void_p]),
    ("srv_submit", c_uint32, [c_void_p, POINTER(_Query), c_void_p, c_size_t, POINTER(c_uint64)]),
    ("srv_completion_arrays", c_uint32, [c_void_p, POINTER(POINTER(c_uint64)), POINTER(POINTER(c_uint64)),
                                         POINTER(POINTER(c_uint64)), POINTER(c_uint32)]),
    ("srv_stop", c_uint32, [c_void_p]),
    ("srv_idle_limit", c_uint32, [c_void_p, c_uint64]),
    ("srv_heartbeat", c_uint32, [c_void_p]),
    ("srv_request_stop", c_uint32, [c_void_p]),
    ("srv_destroy", c_uint32, [c_void_p]),
    ("sssp_run_noalloc", c_uint32, [POINTER(_Csr), c_void_p, c_uint32, c_void_p, POINTER(_Opts), c_void_p]),
    ("pbh_last_error", c_char_p, []),
    ("pbh_version", c_char_p, []),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libpbh.so (raises if it is not built; no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"libpbh.so is not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != 0:
        raise PbhError(status, where, _lib.pbh_last_error().decode(errors="replace"))


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("CUDA device required (no CPU path exists)")
    return torch


def _stream(torch, device=None):
    return c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t) -> c_void_p:
    return c_void_p(t.data_ptr())


def _as_dev_u32(torch, a, device):
    if isinstance(a, np.ndarray):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).to(device)
    assert a.dtype == torch.int32 and a.is_cuda and a.is_contiguous()
    return a


def _to_u64(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def _to_u32(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


# ------------------------------------------------------------------ heap

class Heap:
    """parBucketHeap on one GPU (Section 2.2).

    bulk_update(keys, prios): BulkUpdate of <= d (key, priority) pairs.
    extract_min(r): the min(r, size) smallest elements, ascending (prio, key).
    """

    def __init__(self, key_space: int, d: int, capacity: int = 0, device=None):
        torch = _torch()
        lib = load()
        self.torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.key_space, self.d = key_space, d
        self._params = _Params(key_space, d, capacity)
        nbytes = lib.pbh_workspace_bytes(byref(self._params))
        if nbytes == 0:
            raise PbhError(1, "pbh_workspace_bytes", "invalid parameters")
        self.workspace_bytes = nbytes
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._h = c_void_p()
        _check(lib.pbh_create(byref(self._h), byref(self._params), _ptr(self.ws), nbytes,
                              _stream(torch, self.device)), "pbh_create")
        self.keys_out = torch.empty(max(d, 1), dtype=torch.int32, device=self.device)
        self.prios_out = torch.empty(max(d, 1), dtype=torch.int32, device=self.device)
        self.count_out = torch.zeros(1, dtype=torch.int32, device=self.device)

    def bulk_update(self, keys, prios) -> None:
        k = _as_dev_u32(self.torch, keys, self.device)
        p = _as_dev_u32(self.torch, prios, self.device)
        assert k.numel() == p.numel()
        _check(_lib.pbh_bulk_update(self._h, _ptr(k), _ptr(p), k.numel()), "pbh_bulk_update")
        self._keep = (k, p)  # keep inputs alive until the stream consumes them

    def assign(self, keys, prios) -> None:
        """pbh_assign: general update, the last pair of a key wins (up or down)."""
        k = _as_dev_u32(self.torch, keys, self.device)
        p = _as_dev_u32(self.torch, prios, self.device)
        assert k.numel() == p.numel()
        _check(_lib.pbh_assign(self._h, _ptr(k), _ptr(p), k.numel()), "pbh_assign")
        self._keep = (k, p)

    def delete(self, keys) -> None:
        """pbh_delete: every listed live key stops being live."""
        k = _as_dev_u32(self.torch, keys, self.device)
        _check(_lib.pbh_delete(self._h, _ptr(k), k.numel()), "pbh_delete")
        self._keep = (k,)

    def extract_min_async(self, r: int):
        """Enqueue extract; returns device tensors (keys, prios, count[1])."""
        _check(_lib.pbh_extract_min(self._h, r, _ptr(self.keys_out), _ptr(self.prios_out),
                                    _ptr(self.count_out)), "pbh_extract_min")
        return self.keys_out, self.prios_out, self.count_out

    def extract_min(self, r: int):
        """Extract and return host arrays (keys uint32, prios uint32)."""
        k, p, c = self.extract_min_async(r)
        n = int(c.item())
        return _to_u32(k[:n]), _to_u32(p[:n])

    def ops_array(self, ops, outs=None):
        """The pbh_op array of a sequence.  ops: ("bulk", keys, prios) with
        int32 device tensors, or ("extract", r).  outs (optional) reuses output
        tensors, one (keys, prios, count[1]) per extract.  Returns (array,
        outs, tensors to keep alive)."""
        torch = self.torch
        arr = (_Op * max(len(ops), 1))()
        new_outs, keep, e = [], [], 0
        for i, op in enumerate(ops):
            if op[0] == "bulk":
                k = _as_dev_u32(torch, op[1], self.device)
                p = _as_dev_u32(torch, op[2], self.device)
                keep += [k, p]
                arr[i] = _Op(OP_BULK_UPDATE, k.numel(), 0, 0, k.data_ptr(), p.data_ptr(), None, None, None)
            else:
                r = int(op[1])
                if outs is not None:
                    ko, po, co = outs[e]
                else:
                    ko = torch.empty(max(r, 1), dtype=torch.int32, device=self.device)
                    po = torch.empty(max(r, 1), dtype=torch.int32, device=self.device)
                    co = torch.zeros(1, dtype=torch.int32, device=self.device)
                e += 1
                new_outs.append((ko, po, co))
                arr[i] = _Op(OP_EXTRACT, 0, r, 0, None, None, ko.data_ptr(), po.data_ptr(), co.data_ptr())
        return arr, new_outs, keep

    def run_ops(self, ops, deep_ctas: int = 128, outs=None, arr=None):
        """pbh_run_ops: a sequence of operations in one launch (per 4096) with
        concurrent level resolution (deep_ctas CTAs for Resolve(2) and deeper;
        0 = phase by phase).  Returns, per extract, device tensors (keys,
        prios, count[1]) holding its result."""
        if arr is None:
            arr, outs, keep = self.ops_array(ops, outs)
            self._keep = keep
        _check(_lib.pbh_run_ops(self._h, arr, len(ops), int(deep_ctas)), "pbh_run_ops")
        return outs

    def size(self) -> int:
        out = c_uint64()
        _check(_lib.pbh_size(self._h, byref(out)), "pbh_size")
        return int(out.value)

    def sync(self) -> None:
        _check(_lib.pbh_sync(self._h), "pbh_sync")

    def stats(self) -> dict:
        """Counters since creation (merged, stale_dropped, resolves, barriers, phase times)."""
        st = _Stats()
        _check(_lib.pbh_stats(self._h, byref(st)), "pbh_stats")
        out = {k: getattr(st, k) for k in ("merged", "stale_dropped", "barriers", "t_sort_ns", "t_empty0_ns",
                                            "t_fill0_ns", "t_deeper_ns", "t_ensure_ns")}
        out["resolves"] = list(st.resolves)
        return out

    def validate(self):
        v, s = c_uint32(), c_uint64()
        _check(_lib.pbh_validate(self._h, byref(v), byref(s)), "pbh_validate")
        return int(v.value), int(s.value)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.pbh_destroy(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ SSSP

class DeviceGraph:
    """CSR arrays resident on the GPU (row_ptr as int64, col / w as int32)."""

    def __init__(self, g, device=None):
        torch = _torch()
        self.n, self.m = int(g.n), int(g.m)
        self.name = getattr(g, "name", "")
        dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.row_ptr = torch.from_numpy(np.ascontiguousarray(g.row_ptr, dtype=np.uint64).view(np.int64)).to(dev)
        col = np.ascontiguousarray(g.col, dtype=np.uint32)
        w = np.ascontiguousarray(g.w, dtype=np.uint32)
        self.col = torch.from_numpy((col if len(col) else np.zeros(1, np.uint32)).view(np.int32)).to(dev)
        self.w = torch.from_numpy((w if len(w) else np.zeros(1, np.uint32)).view(np.int32)).to(dev)
        self.max_degree = int(np.max(np.diff(g.row_ptr.astype(np.int64)))) if self.n else 0
        self.device = dev

    @property
    def nbytes(self) -> int:
        return 8 * (self.n + 1) + 8 * self.m

    def csr(self) -> _Csr:
        return _Csr(self.n, self.m, self.row_ptr.data_ptr(), self.col.data_ptr())


def _opts(r=0, d=0, cta=0, flags=0, limit_ms=0, wait_us=0):
    return _Opts(int(r), int(d), int(cta), int(flags), int(limit_ms), int(wait_us))


class SsspWorkspace:
    """Device workspace for sssp_run, reusable across runs of one size.
    auto=True passes no options: the library picks the team by graph size."""

    def __init__(self, n: int, r=0, d=0, cta=0, device=None, flags=0, limit_ms=0, wait_us=0, auto=False):
        torch = _torch()
        lib = load()
        self.opts = _opts(r, d, cta, flags, limit_ms, wait_us)
        self.auto = auto
        self.bytes = lib.sssp_workspace_bytes(n, None if auto else byref(self.opts))
        if self.bytes == 0:
            raise PbhError(1, "sssp_workspace_bytes", "invalid options")
        self.buf = torch.empty(self.bytes, dtype=torch.uint8, device=device or "cuda")


def sssp_async(dg: DeviceGraph, source: int, dist=None, ws: SsspWorkspace | None = None, r=0, d=0, cta=0, flags=0,
               limit_ms=0, wait_us=0, auto=False):
    """Enqueue sssp_run; returns (dist int64 tensor with uint64 bits, workspace)."""
    torch = _torch()
    lib = load()
    if ws is None:
        ws = SsspWorkspace(dg.n, r, d, cta, dg.device, flags=flags, limit_ms=limit_ms, wait_us=wait_us, auto=auto)
    if dist is None:
        dist = torch.empty(max(dg.n, 1), dtype=torch.int64, device=dg.device)
    csr = dg.csr()
    _check(lib.sssp_run(byref(csr), _ptr(dg.w), source, _ptr(dist), None if ws.auto else byref(ws.opts), _ptr(ws.buf),
                        ws.bytes, _stream(torch, dg.device)), "sssp_run")
    return dist, ws


def sssp_stats(ws: SsspWorkspace) -> dict:
    torch = _torch()
    st = _Stats()
    status = _lib.sssp_stats(_ptr(ws.buf), byref(st), _stream(torch, ws.buf.device))
    out = {k: getattr(st, k) for k in ("rounds", "extracted", "relaxations", "improvements", "stale_dropped",
                                        "merged", "levels", "r_eff", "max_degree", "status", "t_relax_ns",
                                        "t_sort_ns", "t_empty0_ns", "t_fill0_ns", "t_deeper_ns", "t_ensure_ns",
                                        "barriers", "settled")}
    out["resolves"] = list(st.resolves)[: max(out["levels"], 1)]
    if status != 0:
        raise PbhError(status, "sssp (device)", _lib.pbh_last_error().decode(errors="replace"))
    return out


def sssp(dg: DeviceGraph, source: int, r=0, d=0, cta=0, with_stats=False, flags=0, limit_ms=0, wait_us=0, auto=False):
    """Exact distances as a numpy uint64 array (UINT64_MAX = unreachable).
    auto=True leaves the options to the library (team chosen by graph size)."""
    dist, ws = sssp_async(dg, source, r=r, d=d, cta=cta, flags=flags, limit_ms=limit_ms, wait_us=wait_us, auto=auto)
    st = sssp_stats(ws)  # synchronises and raises on a latched device error
    out = _to_u64(dist[: dg.n])
    return (out, st) if with_stats else out


def sssp_host(g, source: int, r=0, d=0, cta=0, ws=None, pinned=None, flags=0):
    """sssp_run_host: host CSR in, host distances out (copies inside the call)."""
    torch = _torch()
    lib = load()
    opts = _opts(r, d, cta, flags)
    n, m = int(g.n), int(g.m)
    need = lib.sssp_host_workspace_bytes(n, m, byref(opts))
    if ws is None or ws.numel() < need:
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    if pinned is None:
        pinned = HostBuffers(g)
    _check(lib.sssp_run_host(n, m, pinned.row_ptr.ctypes.data, pinned.col.ctypes.data, pinned.w.ctypes.data, source,
                             pinned.dist.ctypes.data, byref(opts), _ptr(ws), need, _stream(torch)), "sssp_run_host")
    return pinned.dist, ws


class HostBuffers:
    """Pinned host copies of a graph plus a pinned distance array."""

    def __init__(self, g):
        torch = _torch()

        def pin(a, dt):
            t = torch.from_numpy(np.ascontiguousarray(a).view(dt)).pin_memory()
            self._keep.append(t)
            return t.numpy()

        self._keep = []
        self.row_ptr = pin(g.row_ptr, np.int64)
        self.col = pin(g.col if len(g.col) else np.zeros(1, np.uint32), np.int32)
        self.w = pin(g.w if len(g.w) else np.zeros(1, np.uint32), np.int32)
        d = torch.empty(max(int(g.n), 1), dtype=torch.int64).pin_memory()
        self._keep.append(d)
        self.dist = d.numpy().view(np.uint64)

    @property
    def h2d_bytes(self) -> int:
        return self.row_ptr.nbytes + self.col.nbytes + self.w.nbytes

    @property
    def d2h_bytes(self) -> int:
        return self.dist.nbytes


# ---------------------------------------------------------------- batched

class Batch:
    """Many independent queries in one persistent launch (sssp_batch_run)."""

    def __init__(self, graphs, sources, r=0, d=0, cta=0):
        torch = _torch()
        lib = load()
        self.graphs = list(graphs)
        self.sources = list(sources)
        nq = len(self.graphs)
        self.dist = [torch.empty(max(g.n, 1), dtype=torch.int64, device=g.device) for g in self.graphs]
        rs = r if isinstance(r, (list, tuple)) else [r] * nq
        ds = d if isinstance(d, (list, tuple)) else [d] * nq
        cs = cta if isinstance(cta, (list, tuple)) else [cta] * nq
        self.q = (_Query * max(nq, 1))()
        for i, (g, s) in enumerate(zip(self.graphs, self.sources)):
            self.q[i] = _Query(g.csr(), g.w.data_ptr(), int(s), self.dist[i].data_ptr(), int(rs[i]), int(ds[i]),
                               int(cs[i]))
        self.nq = nq
        self.bytes = lib.sssp_batch_workspace_bytes(self.q, nq)
        if nq and self.bytes == 0:
            raise PbhError(1, "sssp_batch_workspace_bytes", "invalid options")
        self.ws = torch.empty(max(self.bytes, 1), dtype=torch.uint8, device="cuda")

    def run_async(self):
        torch = _torch()
        _check(_lib.sssp_batch_run(self.q, self.nq, _ptr(self.ws), self.bytes, _stream(torch)), "sssp_batch_run")

    def status(self):
        torch = _torch()
        st = (c_uint32 * max(self.nq, 1))()
        rounds = (c_uint64 * max(self.nq, 1))()
        code = _lib.sssp_batch_status(_ptr(self.ws), self.nq, st, rounds, _stream(torch))
        return code, list(st)[: self.nq], list(rounds)[: self.nq]

    def run(self):
        self.run_async()
        code, st, rounds = self.status()
        if code != 0:
            raise PbhError(code, "sssp_batch (device)", f"per-query status {st}")
        return [_to_u64(d[: g.n]) for d, g in zip(self.dist, self.graphs)]
