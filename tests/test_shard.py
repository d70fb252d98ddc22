"""Sharding of environment batches over ranks (the N > 1 benchmark path),
on CPU: the cost-balanced partition, per-rank seeds, the timing reduction
over two gloo ranks, and each rank's slice of the benchmark's batch."""
import os
import socket

import numpy as np
import pytest

from paper_2507_01152_gb300 import scene, shard

torch = pytest.importorskip("torch")


def test_partition_covers_every_env_once_and_balances_cost():
    probes = scene.c3_probes()
    rng = np.random.default_rng(4)
    envs = np.stack([np.zeros(97), rng.integers(0, 3, 97)], axis=1).astype(np.int32)
    costs = shard.env_costs(probes, envs)
    for world in (1, 2, 3, 8):
        parts = shard.partition(costs, world)
        assert len(parts) == world and parts[0][0] == 0 and parts[-1][1] == len(envs)
        assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))          # contiguous, no gap, no overlap
        loads = [costs[lo:hi].sum() for lo, hi in parts]
        assert max(loads) - min(loads) <= 2 * costs.max()                  # within two envs of each other


def test_partition_edge_cases():
    assert shard.partition([], 3) == [(0, 0)] * 3
    assert shard.partition([5.0], 2) in ([(0, 1), (1, 1)], [(0, 0), (0, 1)])
    assert shard.partition([1.0] * 8, 4) == [(0, 2), (2, 4), (4, 6), (6, 8)]
    with pytest.raises(ValueError):
        shard.partition([1.0], 0)


def test_env_costs_match_probe_sizes():
    probes = [scene.linear_probe(8, 16, 8.0, 0.5), scene.curvilinear_probe(16, 32, 10.0, 60.0, 5.0, 20, 10)]
    c = shard.env_costs(probes, np.array([[0, 1], [0, 0]], np.int32))
    assert list(c) == [16 * 32 + 20 * 10, 8 * 16 + 16 * 8]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        wl = bench.make_workload("paper", world)            # global batch of `world` per-rank batches
        sub, (lo, hi) = bench.rank_workload(wl, rank, world)
        secs, units = shard.reduce_timing(0.1 * (rank + 1), len(sub.envs) * 3, dist)
        span = torch.tensor([lo, hi], dtype=torch.int64)
        spans = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(spans, span)
        q.put((rank, secs, units, [tuple(int(v) for v in s_) for s_ in spans], shard.rank_seed(wl.seed, rank),
               len(wl.envs), np.array_equal(sub.poses, wl.poses[lo:hi])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_batch_and_reduce_timing():
    import torch.multiprocessing as mp
    with socket.socket() as s_:
        s_.bind(("127.0.0.1", 0))
        port = s_.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, u0, sp0, seed0, n0, ok0), (r1, s1, u1, sp1, seed1, n1, ok1) = res
    assert s0 == s1 == pytest.approx(0.2)                 # the slowest rank's time
    assert u0 == u1 == n0 * 3                              # all ranks' units
    assert sp0 == sp1 and sp0[0][0] == 0 and sp0[0][1] == sp0[1][0] and sp0[1][1] == n0
    assert sp0[0][1] - sp0[0][0] == sp0[1][1] - sp0[1][0] == n0 // 2   # equal costs: equal halves
    assert seed0 != seed1 and ok0 and ok1
