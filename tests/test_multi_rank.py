"""The multi-GPU host logic on CPU with the gloo backend, world size 2:
query sharding (every query on exactly one rank, balanced) and the
max-over-ranks timing / sum-over-ranks units reductions bench.py uses."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, weights, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    d = bench.Dist(world, backend="gloo")
    d.init(torch)
    mine = bench.shard(weights, d.rank, d.world)
    t_local = 1.0 + rank          # rank 1 is the slow one
    units = float(sum(weights[i] for i in mine))
    out[rank] = (mine, d.max(torch, t_local), d.sum(torch, units))
    d.barrier(torch)
    d.close()


def test_shard_and_reductions_world2():
    weights = [((i * 7919) % 101) + 1 for i in range(64)]
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, weights, out), nprocs=world, join=True)
        res = dict(out)
    shards = [res[r][0] for r in range(world)]
    assert sorted(shards[0] + shards[1]) == list(range(64))     # each query exactly once
    loads = [sum(weights[i] for i in s) for s in shards]
    assert abs(loads[0] - loads[1]) <= max(weights)            # balanced (greedy LPT)
    for r in range(world):
        assert res[r][1] == 2.0                                  # max over ranks
        assert res[r][2] == float(sum(weights))                  # sum over ranks


def test_shard_single_rank_is_identity():
    assert bench.shard([5, 1, 3], 0, 1) == [0, 1, 2]


def test_bench_spawns_its_own_ranks():
    # `bench.py --gpus 2` outside torchrun starts two ranks itself (torchrun,
    # 127.0.0.1); the host-only "ranks" workload runs them on gloo and rank 0
    # reports the world size and the sharded query count
    import json
    import subprocess
    import sys
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_PORT")}
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--workload", "ranks", "--gpus", "2",
                          "--queries", "64"], capture_output=True, text=True, env=env, timeout=240)
    assert res.returncode == 0, res.stderr[-2000:]
    line = [x for x in res.stdout.splitlines() if x.startswith("{")][-1]
    j = json.loads(line)
    assert j["world"] == 2 and j["queries_total"] == 64
    assert bench.spawn_command(type("A", (), {"gpus": 1})(), []) is None
