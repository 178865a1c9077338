"""Host-side helpers for runs on several GPUs of one node (one process per GPU).

The evaluation of one surface has no exchange step, and independent surfaces share nothing, so a
multi-GPU run either evaluates a replica per rank or splits a batch of surfaces over the ranks:
longest-processing-time-first on a per-surface cost, no data-path collective.  The only
collectives are the timing ones (a barrier and a max over ranks), on whatever backend the process
group uses (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import heapq
import os

import torch


def env():
    """(world_size, rank, local_rank) from the launcher's environment (1, 0, 0 without one)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def lpt_shards(costs, n_ranks):
    """Indices of the items each rank evaluates: items by decreasing cost, each to the currently
    least-loaded rank (ties to the lower rank), every rank's list in increasing index order."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    heap = [(0.0, r) for r in range(n_ranks)]
    shards = [[] for _ in range(n_ranks)]
    for i in order:
        load, r = heapq.heappop(heap)
        shards[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(s) for s in shards]


def max_over_ranks(value, device=None):
    """The largest of every rank's value (the job's time is its slowest rank's); the value itself
    without an initialised process group."""
    import torch.distributed as d

    if not (d.is_available() and d.is_initialized()) or d.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    d.all_reduce(t, op=d.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, device=None):
    """Sum of every rank's value (work done by the whole job)."""
    import torch.distributed as d

    if not (d.is_available() and d.is_initialized()) or d.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    d.all_reduce(t, op=d.ReduceOp.SUM)
    return float(t.item())


def barrier():
    import torch.distributed as d

    if d.is_available() and d.is_initialized() and d.get_world_size() > 1:
        d.barrier()
