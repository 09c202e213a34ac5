"""Instance sharding across ranks (one process per GPU, torch.distributed).

The path shards by instance: rank r contracts a contiguous block of the global
instance list on its own GPU and no data moves between ranks while it runs.
Afterwards results can be gathered (all_gather_object) and the step time is the
maximum over ranks.  These helpers hold no contraction arithmetic.
"""
import torch.distributed as dist


def shard_range(n_total, rank, world):
    """Contiguous [begin, end) block of instance indices owned by `rank`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    base, extra = divmod(n_total, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def gather_results(local, n_total, rank, world):
    """All-gather per-instance results: `local` maps global index -> result.

    Returns a list of n_total results (every rank gets the full list).
    """
    if world == 1:
        out = [None] * n_total
        for k, v in local.items():
            out[k] = v
        return out
    parts = [None] * world
    dist.all_gather_object(parts, dict(local))
    out = [None] * n_total
    for part in parts:
        for k, v in part.items():
            out[k] = v
    return out


def max_over_ranks(value, world, device=None):
    """Largest value over ranks (the slowest rank's time)."""
    if world == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
