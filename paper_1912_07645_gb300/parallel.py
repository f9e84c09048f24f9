"""Monte Carlo samples sharded across GPUs (one process per GPU) and their statistics merged.

Samples are independent (Sec. 2.2), so each rank advances a contiguous range of the ensemble with
no communication on the data path; the only exchange is one all-gather of the per-rank Welford
accumulators at the end, merged in rank order with alsv_stats_merge (Chan-Golub-LeVeque), which
makes the ensemble statistics independent of timing.
"""
from __future__ import annotations


def shard(rank: int, world: int, total: int):
    """Contiguous sample range (first, count) of `rank` among `world` ranks."""
    if world < 1 or not (0 <= rank < world) or total < 0:
        raise ValueError("need 0 <= rank < world and total >= 0")
    base, extra = divmod(total, world)
    first = rank * base + min(rank, extra)
    count = base + (1 if rank < extra else 0)
    return first, count


def gather(t, group=None):
    """All-gather equally sized tensors; returns the list in rank order."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    out = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(out, t.contiguous(), group=group)
    return out


def merge_in_rank_order(solver, gathered):
    """Merge per-rank accumulators (device tensors, rank order) into a fresh accumulator."""
    from . import _abi as A
    torch = solver.torch
    # the all-gather ran on the current stream: the solver's stream must not start before it ends
    solver.stream.wait_stream(torch.cuda.current_stream(solver.device))
    with torch.cuda.stream(solver.stream):
        out = torch.zeros_like(gathered[0])
    for t in gathered:
        A.alsv_stats_merge(solver.ctx, out, t)
    return out
