"""Replica parallelism over several processes (one GPU each).

Replicas are independent (App. B: many replicas evolve in parallel and the
best is kept), so N processes each solve their own replicas with their own
seeds and nothing is exchanged while they run. The only exchanges are after
the run: the longest rank's time (for a throughput over the whole job) and
the best solution over ranks, which is the argmin of (energy, rank) - the
lowest energy, the lowest rank on ties - followed by a broadcast of that
rank's vector. Works on any torch.distributed backend (gloo on the host,
NCCL between GPUs); with no process group it is the identity.
"""
from __future__ import annotations

import numpy as np


def rank_seed(seed: int, rank: int) -> int:
    """Seed of a rank's replicas: disjoint Philox keys per rank."""
    return int(seed) + 1000 * int(rank)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over the ranks of the default group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def best_over_ranks(E: float, x: np.ndarray, dist=None, device=None):
    """(E_best, x_best, rank_best): the lowest energy over the ranks (lowest
    rank on ties) and that rank's vector, on every rank."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(E), np.asarray(x), 0
    import torch
    world, rank = dist.get_world_size(), dist.get_rank()
    allE = torch.zeros(world, dtype=torch.float64, device=device)
    allE[rank] = float(E)
    dist.all_reduce(allE, op=dist.ReduceOp.SUM)          # each rank fills its own slot
    e = allE.cpu().numpy()
    winner = int(np.flatnonzero(e == e.min())[0])
    xt = torch.as_tensor(np.ascontiguousarray(x, dtype=np.uint8), device=device).clone()
    dist.broadcast(xt, src=winner)
    return float(e[winner]), xt.cpu().numpy(), winner
