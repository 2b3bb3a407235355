"""One system's force evaluation split over ranks, one process per GPU.

Every rank holds the whole tree: it builds it from the same positions, masses
and root shift, and the build is deterministic (the same bits on every GPU),
so no tree data moves between ranks.  The active set is cut into contiguous,
balanced ranges of the caller's order; each rank walks its own range, and the
ranges are gathered in rank order.  Each result row belongs to exactly one
rank, so the only exchange is that gather: no reduction.  The same code runs
over NCCL with device tensors and over gloo with host tensors.
"""
from __future__ import annotations


def active_range(n_active: int, rank: int, world: int) -> tuple:
    """Contiguous range [lo, hi) of ``n_active`` items owned by ``rank``; the
    ranges cover [0, n_active) in rank order and differ in size by at most 1."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    if n_active < 0:
        raise ValueError("n_active must be >= 0")
    q, r = divmod(int(n_active), world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def gather_rows(local, n_total: int, rank: int, world: int, group=None):
    """Concatenates every rank's ``local`` rows in rank order (ranks own the
    ranges of ``active_range(n_total, ., world)``).  Slices are padded to the
    largest one for the collective and trimmed afterwards."""
    import torch
    import torch.distributed as dist

    lo, hi = active_range(n_total, rank, world)
    if local.shape[0] != hi - lo:
        raise ValueError("rank %d holds %d rows, its range has %d" % (rank, local.shape[0], hi - lo))
    if world == 1:
        return local
    width = -(-n_total // world)  # the largest range
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[:hi - lo] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    rows = []
    for r in range(world):
        a, b = active_range(n_total, r, world)
        rows.append(parts[r][:b - a])
    return torch.cat(rows)


def sharded_compute_forces(compute, active_ids, rank: int, world: int, group=None):
    """Runs ``compute(ids)`` -- e.g. ``System.compute_forces`` on this rank's
    replica -- on this rank's range of ``active_ids`` and gathers every
    returned per-particle array into the full active order."""
    n = len(active_ids)
    lo, hi = active_range(n, rank, world)
    outs = compute(active_ids[lo:hi])
    return tuple(gather_rows(o, n, rank, world, group) for o in outs)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The largest ``value`` over all ranks (a step time, for instance)."""
    import torch
    import torch.distributed as dist

    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
