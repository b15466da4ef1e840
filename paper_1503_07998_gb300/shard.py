"""Sharding of independent planes or volumes over ranks (one process per GPU).

Planes orthogonal to the rotation axis are deconvolved independently
(Results section), so the path shards with no data-path collective: a rank
takes a contiguous range of planes (strong scaling of one volume) or its own
volumes (weak scaling).  The only collectives are host-side timing ones
(barrier, max over ranks), used by the benchmark.
"""

from __future__ import annotations


def plane_range(n_planes: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous [lo, hi) of the planes rank `rank` of `world` deconvolves;
    the ranges partition [0, n_planes) and differ in size by at most one."""
    if world < 1 or not 0 <= rank < world or n_planes < 0:
        raise ValueError("bad rank/world/planes")
    base, extra = divmod(n_planes, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def volumes_of_rank(n_volumes: int, rank: int, world: int) -> list[int]:
    """Volume indices rank `rank` handles (round robin)."""
    return list(range(rank, n_volumes, world))


def max_over_ranks(x: float) -> float:
    """Max of a host float over the default process group (identity without
    one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
