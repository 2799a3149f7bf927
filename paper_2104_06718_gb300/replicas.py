"""Replica-parallel host logic: one process per GPU, subdomains split by rank.

Subdomains are independent problems (the batch of Sec. 5.2 bounds each one
on its own), so the bounding path shards with no exchange during the
iterations: every rank holds a full copy of the network and bounds a
contiguous block of the subdomain list.  The only exchange is optional and
happens after the bound: gathering every rank's `out` (and its rho_T for
warm starts) to the process that drives branch and bound.

These helpers work on any torch.distributed backend (NCCL between GPUs,
gloo on CPU); none of them runs inside the bounding path.
"""
from __future__ import annotations

import torch


def block_range(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous block [start, start + count) of n_total units owned by
    `rank` of `world`; block sizes differ by at most one, lower ranks first."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError(f"bad partition: n_total={n_total} world={world} rank={rank}")
    base, extra = divmod(n_total, world)
    count = base + (1 if rank < extra else 0)
    start = rank * base + min(rank, extra)
    return start, count


def gather_rows(local: torch.Tensor, n_total: int, group=None) -> torch.Tensor:
    """All-gather of per-rank row blocks (the layout of `block_range`) into
    the full [n_total, ...] tensor on every rank.  Blocks may be ragged (the
    smaller ones are padded for the collective and trimmed afterwards)."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    start, count = block_range(n_total, world, rank)
    if local.shape[0] != count:
        raise ValueError(f"rank {rank} holds {local.shape[0]} rows, its block has {count}")
    width = -(-n_total // world) if world else 0
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[:count] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    rows = []
    for r in range(world):
        _, c = block_range(n_total, world, r)
        rows.append(parts[r][:c])
    return torch.cat(rows, dim=0)


def max_over_ranks(values, device=None, group=None) -> list[float]:
    """Element-wise maximum of a list of floats over all ranks (the step time
    of a replica job is the slowest rank's)."""
    import torch.distributed as dist

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return t.tolist()
