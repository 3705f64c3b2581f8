"""sssp_run_noalloc, the allocation-free entry point, called through the C ABI.

Some callers cannot allocate device memory at the moment they run a query
(a process under a fixed device-memory budget, an allocator that must not
grow, a path where cudaMalloc would stall the device).  For them the library
runs the same query kernel on a static scratch array it owns.  These tests
check that its distances equal those of sssp_run (caller-provided
workspace) exactly -- distances are integers, so the tolerance is zero -- on
two calls in a row: the second call finds the first call's leftovers in the
shared array and must not be affected by them.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu


def _noalloc(lib, dg, source, opts=(0, 0, 0, 0)):
    import torch
    so = lib.load()
    out = torch.full((max(dg.n, 1),), 7, dtype=torch.int64, device="cuda")
    csr = dg.csr()
    o = lib._Opts(*opts)
    status = so.sssp_run_noalloc(ctypes.byref(csr), ctypes.c_void_p(dg.w.data_ptr()), source,
                                 ctypes.c_void_p(out.data_ptr()), ctypes.byref(o),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return status, out[: dg.n].cpu().numpy().view(np.uint64)


def test_noalloc_matches_sssp_run_twice(lib):
    cases = [(gen.banded(1 << 14, 32, 256, 1, 65535, 3), 0, (0, 0, 0, 0)),
             (gen.grid(100, 100, 1, 100, 4), 5050, (64, 1024, 0, 0))]
    for g, source, opts in cases:
        dg = lib.DeviceGraph(g)
        want = lib.sssp(dg, source, r=opts[0], d=opts[1])  # the existing entry point
        status, got = _noalloc(lib, dg, source, opts)
        assert status == 0, lib.load().pbh_last_error()
        assert np.array_equal(got, want)


def test_noalloc_size_limit(lib):
    # with the default options a query of 2^18 vertices fits the 32 MiB
    # scratch and one of 2^19 does not
    g = gen.banded(1 << 18, 4, 16, 1, 9, 2)
    dg = lib.DeviceGraph(g)
    status, got = _noalloc(lib, dg, 0)
    assert status == 0, lib.load().pbh_last_error()
    assert np.array_equal(got, lib.sssp(dg, 0))


def test_noalloc_rejects_oversized_query(lib):
    # 2^19 vertices with the default options need more than the 32 MiB scratch
    g = gen.banded(1 << 19, 4, 16, 1, 9, 1)
    dg = lib.DeviceGraph(g)
    status, _ = _noalloc(lib, dg, 0)
    assert status == 2  # PBH_E_NOMEM
    assert b"static scratch" in lib.load().pbh_last_error()
