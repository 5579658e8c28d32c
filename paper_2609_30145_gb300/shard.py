"""Row sharding across ranks (one process per GPU, one library context each).

Every parameter row is independent, so a batch splits into contiguous shards
with no exchange on the data path; the only communication is gathering the
per-row results (lnL, 8 bytes per row) to the ranks that need them, and the
max of per-rank step times for the benchmark.  Works with any
torch.distributed backend (gloo on CPU, NCCL on GPUs).
"""
from __future__ import annotations

import torch


def shard_rows(n: int, rank: int, world: int) -> slice:
    """Contiguous shard of n rows for `rank` of `world` (sizes differ by at most 1)."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    q, r = divmod(n, world)
    start = rank * q + min(rank, r)
    return slice(start, start + q + (1 if rank < r else 0))


def gather_rows(local: torch.Tensor, n: int, world: int, group=None) -> torch.Tensor:
    """All-gather the per-row results of every shard into the full [n, ...] tensor
    (shards as given by shard_rows).  `local` lives on the backend's device."""
    import torch.distributed as dist

    sizes = [shard_rows(n, k, world).stop - shard_rows(n, k, world).start for k in range(world)]
    m = max(sizes)
    pad = torch.zeros((m,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[:local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:s] for p, s in zip(parts, sizes)], dim=0)


def max_over_ranks(x: float, device=None, group=None) -> float:
    """Maximum of a per-rank scalar (e.g. a step time) over all ranks."""
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
