"""Multi-GPU layouts of the Response: independent replicas or row shards.

Replicas (the paper's l replicated PIR servers, Sec. 3): every rank holds the
whole database and answers its own queries; nothing crosses ranks on the data
path.  Row shards: rank r holds rows [r0, r1) of D and of H
(`qpadl_pir_shard_rows`); every rank answers the same query on its rows and
the answers concatenate in rank order, with no reduction, because answer row
i depends on database row i alone (ans = D qu, Def. 1).

Timing across ranks follows one rule: the job's time is the slowest rank's,
and the job's rate is the units all ranks processed divided by it.
"""
from __future__ import annotations

from . import pir


def shard_rows(rows: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [r0, r1) of the database that `rank` of `world` holds."""
    return pir.qpadl_pir_shard_rows(rows, world, rank)


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest `x` over all ranks (`x` itself without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput: units processed by all ranks / slowest rank's time."""
    if max_seconds <= 0:
        raise ValueError("max_seconds must be positive")
    return units_per_rank * world / max_seconds


def gather_row_shards(ans_shard, dist):
    """Concatenate the ranks' answer shards (1-D tensors, possibly of
    different lengths) in rank order on every rank."""
    import torch
    world = dist.get_world_size()
    n = torch.tensor([ans_shard.numel()], dtype=torch.int64, device=ans_shard.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n)
    sizes = [int(s.item()) for s in sizes]
    m = max(sizes) if sizes else 0
    padded = torch.zeros(m, dtype=ans_shard.dtype, device=ans_shard.device)
    padded[: ans_shard.numel()] = ans_shard
    parts = [torch.zeros_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded)
    return torch.cat([p[:k] for p, k in zip(parts, sizes)])
