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
