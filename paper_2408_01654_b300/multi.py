"""Host logic of the multi-rank runs (one process per GPU).

One bundle-adjustment problem does not shard usefully (its dense pose solve
would be dominated by exchanging S), so a multi-rank run gives every rank its
own independent problems: there is no collective on the data path.  The only
communication is the timing: each rank times its own steps and the job's
throughput is the work of all ranks over the slowest rank's time
(max over ranks, weak scaling).  `shard_problems` splits one list of
independent problems across ranks by their solve cost (the dense pose
factorisation grows as N^3) for runs that divide a fixed batch instead.
"""
from __future__ import annotations

import os


def rank_info() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def problem_seed(rank: int) -> int:
    """Each rank's independent synthetic problem (or batch) is seeded by its rank."""
    return rank


def shard_problems(frames: list[int], world: int) -> list[list[int]]:
    """Indices of the problems each rank solves: longest-processing-time
    greedy on the cost N^3 (largest first onto the least loaded rank, ties to
    the lower rank), every problem exactly once, each rank's list ascending."""
    if world < 1:
        raise ValueError("world size must be >= 1")
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for b in sorted(range(len(frames)), key=lambda q: (-frames[q], q)):
        r = min(range(world), key=lambda x: (load[x], x))
        parts[r].append(b)
        load[r] += float(frames[b]) ** 3
    return [sorted(p) for p in parts]


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks (the job's time is its slowest
    rank's); the value itself with one rank or without a process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, max_ms: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest
    rank's time (weak scaling: per-rank work fixed as ranks are added)."""
    return world * units_per_rank / (max_ms / 1e3)
