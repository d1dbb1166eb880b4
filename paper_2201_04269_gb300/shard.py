"""Sharding of the correlator over ranks (one GPU per rank).

Every (set, t, sink site) is independent and C(t) of a set is the sum over its sink sites,
so ranks split the work with no exchange on the data path: by propagator set (each rank
evaluates whole sets: weak scaling, no collective), or, for one set, by contiguous ranges
of sink sites followed by one all-reduce of the partial C (n_sets x T complex values).
"""
from __future__ import annotations


def site_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [begin, end) share of n items for a rank (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def local_sets(n_sets: int, rank: int, world: int) -> range:
    """Propagator sets evaluated by a rank when ranks split by set."""
    b, e = site_range(n_sets, rank, world)
    return range(b, e)


def allreduce_correlator(C, group=None):
    """Sum partial correlators over ranks in place (complex tensor, any device the
    process group's backend supports)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return C
    view = torch.view_as_real(C) if C.is_complex() else C
    dist.all_reduce(view, op=dist.ReduceOp.SUM, group=group)
    return C
