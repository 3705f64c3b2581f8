"""Host logic of the autotuner's table (no GPU): size classes, the batch
rule (r and d per class, large queries on clusters) and the single-query
table, read from a table file written here."""
import json
from types import SimpleNamespace

import pytest

from paper_1908_09378_gb300 import autotune


@pytest.fixture
def table(tmp_path, monkeypatch):
    def use(entries):
        path = tmp_path / "tuned.json"
        path.write_text(json.dumps({autotune._gpu_name(): entries}))
        monkeypatch.setattr(autotune, "CACHE", str(path))
        monkeypatch.setattr(autotune, "_table", None)
        return path
    yield use
    autotune._table = None


def graph(n, m, max_degree):
    return SimpleNamespace(n=n, m=m, max_degree=max_degree)


def test_size_classes():
    assert autotune.size_class(1 << 12, 4) == "12lo"
    assert autotune.size_class(1 << 12, 9) == "12hi"
    assert autotune.size_class(3, 64) == "10hi"          # clamped below
    assert autotune.size_class(1 << 24, 4) == "20lo"     # and above
    assert autotune.size_class(int(1.5 * (1 << 16)), 32) == "17hi"  # rounded log2


def test_d_is_the_next_power_of_two_times_the_multiplier():
    assert autotune.d_for(128, 64) == 8192
    assert autotune.d_for(100, 64) == 8192          # 6400 -> 8192
    assert autotune.d_for(100, 64, 4) == 32768
    assert autotune.d_for(1, 0) == 1


def test_defaults_without_a_table(table):
    table({})
    assert autotune.r_for(1 << 20, 64) == autotune.DEFAULT_R[20]
    assert autotune.teams() == (8, 1 << 22)
    # single queries: a 16-CTA cluster up to 2^19 arcs, else the whole GPU
    assert autotune.single_params(4096, 16128, 4) == (16, 512, 1 << 16)
    assert autotune.single_params(1 << 20, 1 << 26, 64) == (0, 512, 1 << 16)


def test_batch_rule_from_the_table(table):
    table({"12lo": 256, "18hi": {"r": 128, "dmul": 2}, "batch_teams": [4, 1 << 20]})
    gs = [graph(1 << 12, 1 << 14, 4), graph(1 << 18, 1 << 21, 32), graph(1 << 18, 1 << 19, 32)]
    rs, ds, cs = autotune.batch_params(gs)
    assert rs == [256, 128, 128]
    assert ds == [1024, 8192, 8192]  # 256*4 -> 1024; 128*32 = 4096, times 2
    assert cs == [1, 4, 1]            # only the query of >= 2^20 arcs on a 4-CTA cluster
    # a team rule given by the caller wins over the table's
    assert autotune.batch_params(gs, team=(0, 0))[2] == [1, 1, 1]


def test_single_table(table):
    table({"single": {"20hi": {"cta": 0, "r": 384, "d": 65536, "ms": 63.0},
                      "12lo": {"cta": 16, "r": 512, "d": 131072, "ms": 1.5}}})
    assert autotune.single_params(1 << 20, 1 << 26, 64) == (0, 384, 65536)
    assert autotune.single_params(4096, 16128, 4) == (16, 512, 131072)
    assert "20hi" in autotune.describe_single(1 << 20, 64)
    assert "no tuned entry" in autotune.describe_single(1 << 14, 64)


def test_an_unreadable_table_means_defaults(table):
    path = table({})
    path.write_text("{not json")
    assert autotune.r_for(1 << 12, 4) == autotune.DEFAULT_R[12]


def test_team_params(table):
    # a fixed team takes the single-query tuner's best on that team; one CTA,
    # or a team the tuner did not time, takes the batch rule (r, d * mul)
    table({"20hi": {"r": 128, "dmul": 2},
           "single_teams": {"20hi": {"16": {"r": 256, "d": 2097152, "ms": 81.8},
                                     "0": {"r": 384, "d": 2097152, "ms": 60.9}}}})
    assert autotune.team_params(1 << 20, 64, 16) == (256, 2097152)
    assert autotune.team_params(1 << 20, 64, 0) == (384, 2097152)
    assert autotune.team_params(1 << 20, 64, 8) == (128, 16384)   # 128 * 64 = 8192, times 2
    assert autotune.team_params(1 << 20, 64, 1) == (128, 16384)
