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


# ---------------------------------------------------------------------------
# Row-block split of one product (strong scaling): the products of Section 3.1
# split by rows of A and C with no exchange between ranks.  Rank r takes rows
# [m0, m1) of A and the whole of B (replicated: every rank holds its own copy
# in its own GPU's memory) and computes the same rows of C = A B; the only
# communication is the final gather of C's row blocks to rank 0 on the host.
# ---------------------------------------------------------------------------

def row_block(M: int, world_size: int, rank: int):
    """Rows [m0, m1) of rank `rank`: M split as evenly as possible, the first
    M mod world_size ranks taking one row more."""
    if world_size < 1 or not (0 <= rank < world_size) or M < 0:
        raise ValueError("bad split")
    q, r = divmod(M, world_size)
    m0 = rank * q + min(rank, r)
    return m0, m0 + q + (1 if rank < r else 0)


def split_product(A, B, product, world_size: int, rank: int, root: int = 0, group=None):
    """C = A B with the rows of A and C split over the ranks.

    A: [M, K, Wa] words (numpy, the whole matrix or at least this rank's rows),
    B: [K, N, Wb] words, replicated.  ``product(A_rows, B)`` computes this
    rank's row block of C (on this rank's GPU in the bench, any exact product
    in tests) and returns [m1 - m0, N, Wc] uint64 words.  The row blocks are
    gathered to ``root`` over ``torch.distributed`` (host tensors; blocks
    padded to the largest block); root returns the whole C, the other ranks
    their own block.  One rank: just the product."""
    import numpy as np

    M = A.shape[0]
    m0, m1 = row_block(M, world_size, rank)
    block = np.ascontiguousarray(product(A[m0:m1], B), dtype=np.uint64)
    if world_size <= 1:
        return block
    import torch
    import torch.distributed as dist

    rows = max(row_block(M, world_size, r)[1] - row_block(M, world_size, r)[0] for r in range(world_size))
    pad = np.zeros((rows,) + block.shape[1:], dtype=np.uint64)
    pad[: block.shape[0]] = block
    t = torch.from_numpy(pad.view(np.int64))
    parts = [torch.empty_like(t) for _ in range(world_size)] if rank == root else None
    dist.gather(t, gather_list=parts, dst=root, group=group)
    if rank != root:
        return block
    out = []
    for r in range(world_size):
        a, b = row_block(M, world_size, r)
        out.append(parts[r].numpy().view(np.uint64)[: b - a])
    return np.concatenate(out, axis=0)
