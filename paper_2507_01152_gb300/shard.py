"""Sharding of a batch of environments over ranks (one process per GPU).

Environments are independent, so a batch splits into contiguous ranges of
environments, one per rank, with no exchange on the data path: each rank
renders its range into its own frame buffer.  Ranges are balanced by the
render cost of an environment (beam samples plus output pixels of its
probe).  The only collective is the timing reduction of a benchmark: the
slowest rank's time and the units all ranks processed.
"""
from __future__ import annotations

import numpy as np


def env_costs(probes, envs) -> np.ndarray:
    """Cost of rendering each environment: beam samples + output pixels."""
    envs = np.asarray(envs, np.int64).reshape(-1, 2)
    per_probe = np.array([p.n_lines * p.n_samples + p.out_w * p.out_h for p in probes], np.int64)
    return per_probe[envs[:, 1]] if len(envs) else np.zeros(0, np.int64)


def partition(costs, world: int):
    """Contiguous ranges [start, end) of environments, one per rank, cutting
    the running cost where it first reaches k / world of the total.  Every
    environment lands in exactly one range; ranges may be empty when there
    are fewer environments than ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, np.float64)
    n = len(costs)
    if n == 0:
        return [(0, 0)] * world
    cum = np.concatenate([[0.0], np.cumsum(costs)])
    total = cum[-1]
    cuts = [0]
    for k in range(1, world):
        target = total * k / world
        # first boundary whose prefix cost reaches the target, never before
        # the previous cut
        c = int(np.searchsorted(cum, target, side="left"))
        c = min(max(c, cuts[-1]), n)
        # the closer of the two boundaries around the target
        if c > cuts[-1] and abs(cum[c - 1] - target) < abs(cum[c] - target):
            c -= 1
        cuts.append(c)
    cuts.append(n)
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def rank_seed(seed: int, rank: int) -> int:
    """Speckle seed of a rank's replica: every rank draws fresh noise."""
    return int(seed) + 7919 * int(rank)


def reduce_timing(seconds: float, units: int, dist=None, device=None):
    """(max seconds over ranks, total units over ranks): the job's time is
    its slowest rank's, its throughput is all units over that time."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(seconds), int(units)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([int(units)], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())
