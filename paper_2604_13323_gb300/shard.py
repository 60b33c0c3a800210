"""Sharding one batch over several GPUs (one process per GPU).

Every configuration, segment point and VJP row is independent, so a batch
splits across ranks with no exchange during compute: each rank loads the
same robot, constraints and obstacles, projects its part, and the parts are
gathered once at the end (host side).  Two partitions:

  * a plain batch: contiguous ranges of configurations, sizes differing by at
    most one;
  * uneven geodesic segments: contiguous runs of whole segments, cut where
    the running sum of their lengths is nearest to k / world of the total,
    so that every rank projects about the same number of points and no
    segment is split (its points stay in one persistent launch).

A configuration's result does not depend on which other configurations share
the launch (each is projected by its own lane or lane group, every reduction
inside it in a fixed order), so the gathered arrays are identical, bit for
bit, to those of the unsharded run.  The gather is one all_gather per output
array after the compute, through torch.distributed: host tensors under gloo,
staged through the rank's GPU under NCCL.
"""
from __future__ import annotations

import numpy as np


def batch_ranges(n: int, world: int) -> list[tuple[int, int]]:
    """Contiguous [start, stop) ranges of n configurations over `world` ranks."""
    if world < 1 or n < 0:
        raise ValueError("need world >= 1 and n >= 0")
    base, extra = divmod(n, world)
    out, s = [], 0
    for r in range(world):
        e = s + base + (1 if r < extra else 0)
        out.append((s, e))
        s = e
    return out


def segment_ranges(lengths, world: int) -> list[tuple[int, int]]:
    """Contiguous [first, stop) runs of whole segments over `world` ranks,
    balanced by the sum of their lengths: rank r's run ends at the segment
    boundary nearest to (r + 1) / world of the total number of points."""
    lengths = np.asarray(lengths, dtype=np.int64)
    if world < 1 or (lengths < 0).any():
        raise ValueError("need world >= 1 and non-negative lengths")
    S = lengths.size
    cum = np.concatenate([[0], np.cumsum(lengths)])   # cum[k] = points before segment k
    total = int(cum[-1])
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        k = int(np.searchsorted(cum, target))         # first boundary at or above the target
        if k > 0 and abs(cum[k - 1] - target) <= abs(cum[min(k, S)] - target):
            k -= 1
        cuts.append(min(max(k, cuts[-1]), S))
    cuts.append(S)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def point_ranges(lengths, seg_ranges) -> list[tuple[int, int]]:
    """The [start, stop) ranges of segment points (in the unsharded output's
    order) that the runs of whole segments cover."""
    cum = np.concatenate([[0], np.cumsum(np.asarray(lengths, dtype=np.int64))])
    return [(int(cum[a]), int(cum[b])) for a, b in seg_ranges]


def gather_columns(parts, ranges, n_total, group=None):
    """Gathers per-rank column blocks to every rank (host tensors).

    parts: this rank's arrays, each [..., stop - start] for its range (numpy
    or torch; moved to the host).  ranges: every rank's [start, stop).
    Returns the full arrays [..., n_total] in the unsharded order.  With one
    rank, or without an initialised process group, the parts are returned as
    they are."""
    import torch
    import torch.distributed as dist
    hosted = [torch.as_tensor(np.asarray(p.cpu() if hasattr(p, "cpu") else p)) for p in parts]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return [h.numpy() for h in hosted]
    world = dist.get_world_size(group)
    width = max(b - a for a, b in ranges)
    # NCCL moves device buffers only: stage through this rank's GPU
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else None
    out = []
    for h in hosted:
        pad = torch.zeros(h.shape[:-1] + (width,), dtype=h.dtype, device=dev)
        pad[..., :h.shape[-1]] = h.to(pad.device)
        bufs = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(bufs, pad, group=group)
        full = torch.empty(h.shape[:-1] + (n_total,), dtype=h.dtype)
        for (a, b), buf in zip(ranges, bufs):
            full[..., a:b] = buf[..., :b - a].cpu()
        out.append(full.numpy())
    return out
