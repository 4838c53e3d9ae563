"""Scene integration across ranks: the partial images of sub-cubes held by
different processes (one GPU each) combined into the views' images.

The paper distributes the sub-cubes of a cube over GPUs, each renders its
sub-cube into a partial image at screen resolution, and scene integration
combines the partial images (§3.1 items 1, 4, 5; read as the compositing
operator applied in each ray's visibility order).  Here rank r holds
sub-cube r, the cells [cell_lo[r], cell_lo[r + 1]) along z in ascending
order, and its partial images (rendered from an empty start, e.g. with
``Volume.render_part`` and sweep 0).  The exchange is one collective:

  * MIP: an all-reduce with MAX (the maximum needs no order);
  * SUM: an all-reduce with SUM;
  * composite: an all-gather of the partial images, then, on every rank
    (or the root only), the front-to-back "over" of the gathered partials
    in each ray's order -- ascending z when the ray goes up, descending
    otherwise -- by the library's integration kernel
    (``vr_integrate_partials``).

The collectives are torch.distributed's (NCCL between GPUs: plain
device-to-device transfers); the arithmetic of the combination is the
library's kernel.  ``combine`` replaces that kernel only for tests that
check the host-side logic on CPU ranks (gloo), where no kernel can run.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

from .api import integrate_partials


def exchange_partials(partial: torch.Tensor, cams: np.ndarray, mode: str, group=None,
                      root: int | None = None, combine=None) -> torch.Tensor | None:
    """Combine this rank's partial images (views, h, w[, 4]) with the other
    ranks' into the views' images.  Rank r holds sub-cube r (ascending z).
    Returns the images on every rank (``root`` None) or on rank ``root``
    only (None elsewhere)."""
    if mode not in ("mip", "sum", "composite"):
        raise ValueError("unknown mode %r" % mode)
    partial = partial.contiguous()
    rank = dist.get_rank(group)
    world = dist.get_world_size(group)
    if mode in ("mip", "sum"):
        out = partial.clone()
        op = dist.ReduceOp.MAX if mode == "mip" else dist.ReduceOp.SUM
        if root is None:
            dist.all_reduce(out, op=op, group=group)
            return out
        dist.reduce(out, dst=root, op=op, group=group)
        return out if rank == root else None
    if root is None:
        parts = [torch.empty_like(partial) for _ in range(world)]
        dist.all_gather(parts, partial, group=group)
    else:
        parts = [torch.empty_like(partial) for _ in range(world)] if rank == root else None
        dist.gather(partial, parts, dst=root, group=group)
        if rank != root:
            return None
    stacked = torch.stack(parts)                       # (sub-cubes, views, h, w, 4)
    if combine is not None:
        return combine(stacked, cams, mode)
    return integrate_partials(stacked, cams, mode)
