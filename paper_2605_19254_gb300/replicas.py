"""Replica (weak-scaling) bookkeeping for one process per GPU.

The RNS product of Section 3.1 has no exchange step between independent
products: each rank computes its own product on its own GPU, and the only
collective is the timing reduction that turns per-rank step times into one
whole-job throughput.  These helpers hold that bookkeeping so that it can be
exercised on CPU ranks (``gloo``) as well as under ``torchrun`` with NCCL.
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass(frozen=True)
class RankEnv:
    world_size: int
    rank: int
    local_rank: int

    @property
    def is_root(self) -> bool:
        return self.rank == 0


def rank_env(env=None) -> RankEnv:
    """World size, rank and local rank from the torchrun environment (defaults: one rank)."""
    env = os.environ if env is None else env
    ws = int(env.get("WORLD_SIZE", "1"))
    rank = int(env.get("RANK", "0"))
    local = int(env.get("LOCAL_RANK", str(rank)))
    if ws < 1 or not (0 <= rank < ws) or local < 0:
        raise ValueError(f"bad rank environment: WORLD_SIZE={ws} RANK={rank} LOCAL_RANK={local}")
    return RankEnv(ws, rank, local)


def rank_seed(seed: int, rank: int) -> int:
    """Seed of the independent product a rank computes (distinct per rank)."""
    return seed + rank


def max_over_ranks(value: float, world_size: int, device=None) -> float:
    """The largest of every rank's ``value`` (identity for one rank)."""
    if world_size <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world_size: int, seconds_max: float) -> float:
    """Units all ranks processed per second, timed by the slowest rank."""
    if seconds_max <= 0:
        raise ValueError("time must be positive")
    return units_per_rank * world_size / seconds_max
