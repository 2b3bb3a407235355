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


def active_range(n_active: int, rank: int, world: int, weights=None) -> tuple:
    """Contiguous range [lo, hi) of ``n_active`` items owned by ``rank``; the
    ranges cover [0, n_active) in rank order.  Without ``weights`` they
    differ in size by at most 1.  With ``weights`` (one per item, the same on
    every rank -- e.g. each particle's interaction count from the previous
    step, the paper's cost factor of Sec. 8) they hold nearly equal total
    weight: rank r's range ends at the first item whose running sum reaches
    (r + 1) / world of the total, so a rank's weight exceeds its share by
    less than one item's."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside a world of %d" % (rank, world))
    if n_active < 0:
        raise ValueError("n_active must be >= 0")
    if weights is not None:
        import numpy as np

        w = np.asarray(weights, dtype=np.float64).reshape(-1)
        if len(w) != n_active:
            raise ValueError("%d weights for %d items" % (len(w), n_active))
        if n_active and (not np.all(np.isfinite(w)) or w.min() < 0):
            raise ValueError("weights must be finite and >= 0")
        c = np.cumsum(w)
        total = float(c[-1]) if n_active else 0.0
        if total > 0:
            cut = lambda k: n_active if k >= world else int(np.searchsorted(c, total * k / world, side="left")) + 1
            lo, hi = (0 if rank == 0 else cut(rank)), cut(rank + 1)
            return min(lo, n_active), min(max(hi, lo), n_active)
    q, r = divmod(int(n_active), world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def gather_rows(local, n_total: int, rank: int, world: int, group=None, weights=None):
    """Concatenates every rank's ``local`` rows in rank order (ranks own the
    ranges of ``active_range(n_total, ., world, weights)``).  Slices are padded
    to the largest one for the collective and trimmed afterwards."""
    import torch
    import torch.distributed as dist

    lo, hi = active_range(n_total, rank, world, weights)
    if local.shape[0] != hi - lo:
        raise ValueError("rank %d holds %d rows, its range has %d" % (rank, local.shape[0], hi - lo))
    if world == 1:
        return local
    ranges = [active_range(n_total, r, world, weights) for r in range(world)]
    width = max(b - a for a, b in ranges)  # the largest range
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[:hi - lo] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    rows = []
    for r, (a, b) in enumerate(ranges):
        rows.append(parts[r][:b - a])
    return torch.cat(rows)


def sharded_compute_forces(compute, active_ids, rank: int, world: int, group=None, weights=None):
    """Runs ``compute(ids)`` -- e.g. ``System.compute_forces`` on this rank's
    replica -- on this rank's range of ``active_ids`` and gathers every
    returned per-particle array into the full active order.  ``weights``
    (the same on every rank) balance the ranges by work instead of count."""
    n = len(active_ids)
    lo, hi = active_range(n, rank, world, weights)
    outs = compute(active_ids[lo:hi])
    return tuple(gather_rows(o, n, rank, world, group, weights) for o in outs)


def max_over_ranks(value: float, device=None, group=None) -> float:
    """The largest ``value`` over all ranks (a step time, for instance)."""
    import torch
    import torch.distributed as dist

    if not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
