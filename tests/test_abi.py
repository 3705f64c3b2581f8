"""CPU checks of the C ABI: the library builds and loads, exports every
symbol include/pbh.h declares, and the host-side size planning behaves.
No CUDA call is made (this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pbh.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


@pytest.fixture(scope="module")
def so():
    from paper_1908_09378_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_parses():
    names = declared_functions()
    for n in ["pbh_create", "pbh_bulk_update", "pbh_extract_min", "pbh_destroy", "sssp_run", "sssp_batch_run"]:
        assert n in names


def test_every_declared_symbol_is_exported(so):
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_binding_covers_header():
    import paper_1908_09378_gb300 as pbh
    bound = {name for name, _, _ in pbh.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_workspace_planning(so):
    import paper_1908_09378_gb300 as pbh
    lib = pbh.load()
    p = pbh._Params(1 << 24, 1 << 16, 0)
    b = lib.pbh_workspace_bytes(ctypes.byref(p))
    # five levels of ping-pong buckets and buffers: 4 d (4^5 - 1) words, plus cur and U
    levels_words = 4 * (1 << 16) * (4 ** 5 - 1)
    assert b >= 8 * (levels_words + (1 << 24))
    assert b < 8 * (levels_words + (1 << 24)) * 1.05
    bad = pbh._Params(0, 1, 0)
    assert lib.pbh_workspace_bytes(ctypes.byref(bad)) == 0
    o = pbh._Opts(1024, 65536, 0, 0)
    assert lib.sssp_workspace_bytes(1 << 20, ctypes.byref(o)) > 0
    assert lib.pbh_version().startswith(b"pbh-gb300")
