"""The multi-rank path on CPU: two gloo ranks shard independent jobs with no
data-path collective, meet at the timing barrier, and report whole-job
throughput from the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2608_14266_gb300 import replicas


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n_jobs, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    info = replicas.rank_info()
    assert (info.rank, info.world) == (rank, world)
    g = replicas.Group(dist)
    mine = replicas.shard(n_jobs, info.rank, info.world)
    g.barrier()
    seconds = 1.0 + rank  # rank 1 is the slowest
    value, slowest = replicas.throughput(len(mine), seconds, g, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    total = g.sum(len(mine))
    dist.destroy_process_group()
    out.put((rank, mine, gathered, value, slowest, total, replicas.scene_rep(rank)))


def test_two_rank_shards_and_timing():
    world, n_jobs = 2, 11
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n_jobs, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    shards = [r[1] for r in res]
    # the shards partition the jobs, and every rank saw the same partition
    assert sorted(shards[0] + shards[1]) == list(range(n_jobs))
    assert not set(shards[0]) & set(shards[1])
    assert all(r[2] == shards for r in res)
    # slowest rank decides: 2 s on every rank; value = per-rank units x world / 2 s
    for rank, mine, _, value, slowest, total, rep in res:
        assert slowest == 2.0
        assert value == pytest.approx(len(mine) * world / 2.0)
        assert total == n_jobs
        assert rep == rank
    assert res[0][6] != res[1][6]


def test_shard_single_rank_and_errors():
    assert replicas.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert replicas.shard(0, 1, 3) == []
    with pytest.raises(ValueError):
        replicas.shard(5, 2, 2)
    info = replicas.rank_info({})
    assert (info.rank, info.world, info.local) == (0, 1, 0)
    g = replicas.Group(None)
    assert g.max(3.5) == 3.5 and g.sum(2) == 2.0
    assert replicas.throughput(10, 2.0, g, 1) == (5.0, 2.0)
