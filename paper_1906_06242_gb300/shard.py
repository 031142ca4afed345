"""Event-range sharding of the chain across ranks (one GPU per rank).

Events are independent, so a batch shards into contiguous event ranges with
no data exchange; offsets are sliced, not rebased (every kernel accepts
offsets[0] != 0), and the columns are shared. The one exchange of the sharded
chain is the sum of the histograms (integer counts add exactly; binary64
weighted sums up to rounding order).
"""
from __future__ import annotations

import numpy as np


def shard_range(n_events: int, rank: int, world: int):
    """Contiguous [a, b) event range of `rank` out of `world` (sizes differ by
    at most one)."""
    base, extra = divmod(int(n_events), int(world))
    a = rank * base + min(rank, extra)
    b = a + base + (1 if rank < extra else 0)
    return a, b


def shard_host_batch(batch, rank: int, world: int):
    """Host batch (the seeded-input object) restricted to this rank's events."""
    from .synth import EventBatch
    a, b = shard_range(batch.n_events, rank, world)
    out = EventBatch(n_events=b - a, jet_offsets=batch.jet_offsets[a:b + 1], mu_offsets=batch.mu_offsets[a:b + 1],
                     el_offsets=batch.el_offsets[a:b + 1], cols=batch.cols, weight=batch.weight[a:b],
                     seed=batch.seed)
    for attr in ("kin_fmt", "btag_fmt"):
        if hasattr(batch, attr):
            setattr(out, attr, getattr(batch, attr))
    return out


def shard_device_batch(db, rank: int, world: int):
    """Device batch (hepacc.DeviceBatch) restricted to this rank's events;
    the column tensors are shared, offsets and weights are views."""
    from .hepacc import DeviceBatch
    a, b = shard_range(db.n_events, rank, world)
    offs = {k: v[a:b + 1] for k, v in db.offsets.items()}
    return DeviceBatch(b - a, offs, db.cols, db.weight[a:b])


def allreduce_histograms(tensors, group=None):
    """Sum histogram tensors (counts, sumw, sumw2) over the ranks in place."""
    import torch.distributed as dist
    for t in tensors:
        if t is not None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return tensors


__all__ = ["shard_range", "shard_host_batch", "shard_device_batch", "allreduce_histograms"]
