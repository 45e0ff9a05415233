"""Multi-GPU placement of independent contractions (one process per GPU).

Networks are independent units: rank r of a world of w takes every w-th unit
(round robin), so no data-path collective exists.  The only exchange is the
timing reduction a benchmark needs: the maximum of the ranks' elapsed times.

One sliced network (Sec. 4.2.2) splits into 2^s independent slices: each rank
contracts a contiguous slice range, and the ranks' results are added in the
element type (tn.tn_result_combine) -- a max / sum of one scalar per rank.
"""
from __future__ import annotations


def shard(units: int, rank: int, world: int) -> list[int]:
    """Indices of the units rank `rank` runs (round robin)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    return list(range(rank, units, world))


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Maximum of `value` over the ranks of the default process group (the
    value itself when no group is initialised)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def slice_range(nslices: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous slice range [begin, end) of `rank` among `world` ranks for a
    sliced network of `nslices` slices (Sec. 4.2.2); the ranks' results are
    added with tn.tn_result_combine, the one exchange step of the path."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    return nslices * rank // world, nslices * (rank + 1) // world
