"""The multi-rank path on CPU: two gloo ranks shard independent jobs with no
data-path collective, meet at the timing barrier, and report whole-job
throughput from the slowest rank's time; and one job sharded by voxel, whose
iteration needs one all-reduce of the per-scan g, H and the cost."""
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


def _voxel_shard_worker(rank, world, port, out):
    """One large job sharded by voxel: each rank evaluates its voxels (cost
    terms and per-scan g, H partials), one all-reduce sums them, and every
    rank runs the same damped per-scan solves and retraction."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import oracle
    import scenegen
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    s = scenegen.make_scene(scenegen.config("tiny"))
    agg = oracle.points_to_centred(s.point_offsets(), s.points())
    v0, v1 = rank * s.n_voxels // world, (rank + 1) * s.n_voxels // world  # this rank's voxel segment
    o0, o1 = s.voxel_off[v0], s.voxel_off[v1]
    part = oracle.ObsProblem(s.n_scans, s.voxel_off[v0:v1 + 1] - o0, s.obs_scan[o0:o1], agg[o0:o1])
    cost, planes = oracle.voxel_pass(part, s.pose_init)
    g, H = oracle.grad_hess(part, s.pose_init, planes)
    # the iteration's one exchange: n_scans x 27 values and the cost
    buf = torch.from_numpy(np.concatenate([[cost], g.ravel(), H.ravel()]))
    dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    tot = buf.numpy()
    cost, g, H = tot[0], tot[1:1 + 6 * s.n_scans].reshape(-1, 6), tot[1 + 6 * s.n_scans:].reshape(-1, 6, 6)
    mu = oracle.DEFAULT_MU0
    deltas = np.zeros((s.n_scans, 6))
    for j in range(1, s.n_scans):  # scan 0 fixed
        rc, deltas[j] = oracle.ldlt6(H[j] + mu * np.diag(np.diag(H[j])), -g[j])
        assert rc == 0
    trial = oracle.retract_all(s.pose_init, deltas)
    dist.destroy_process_group()
    out.put((rank, cost, g, H, trial))


def test_voxel_sharded_iteration_sums_equal_one_rank():
    """Sharding one job by voxel over two gloo ranks: the all-reduced cost and
    per-scan g, H equal those of the whole problem, and every rank computes
    the same trial poses as the unsharded iteration."""
    import numpy as np

    import oracle
    import scenegen
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_voxel_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=180) for _ in procs], key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    s = scenegen.make_scene(scenegen.config("tiny"))
    full = oracle.ObsProblem(s.n_scans, s.voxel_off, s.obs_scan,
                             oracle.points_to_centred(s.point_offsets(), s.points()))
    cost, planes = oracle.voxel_pass(full, s.pose_init)
    g, H = oracle.grad_hess(full, s.pose_init, planes)
    deltas = np.zeros((s.n_scans, 6))
    for j in range(1, s.n_scans):
        deltas[j] = oracle.ldlt6(H[j] + oracle.DEFAULT_MU0 * np.diag(np.diag(H[j])), -g[j])[1]
    trial = oracle.retract_all(s.pose_init, deltas)
    for _, c_r, g_r, H_r, t_r in res:
        assert c_r == pytest.approx(cost, rel=1e-13)
        np.testing.assert_allclose(g_r, g, rtol=1e-11, atol=1e-13 * np.abs(g).max())
        np.testing.assert_allclose(H_r, H, rtol=1e-11, atol=1e-13 * np.abs(H).max())
        np.testing.assert_allclose(t_r, trial, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(res[0][4], res[1][4])  # identical on every rank
