"""Slab sharding of one data set: x slabs with a halo, one GPU per slab.

A dual cell is emitted by one cell S = (p, l) of width w = 2^l (its owner,
Sec. 4.4: the unique cell that rule 3 lets emit it), and its 8 query points
q = p + d * w, d in {-1, 0, 1}^3, lie within one owner width of p; every
cell snap() returns for q contains q (Sec. 4.2-4.4). A shard holding every
cell that overlaps its slab [x0, x1) grown by the widest cell w_max on both
sides therefore snaps, for owners in the slab, exactly as the whole data set
does: `amr_dual_cells_owned(x0, x1)` on that shard emits exactly the whole
data set's duals owned in the slab, and the slabs together give every dual
once. Marching Cubes on those duals reads only their vertex cells, which the
shard holds, so the triangles are the whole data set's too.

The exchange is the halo itself: each rank uploads its slab plus halo (the
cells it selects from the whole list, here on its own GPU) and extracts
independently; the only collective is the gather of the per-slab counts
(and, when wanted, of the outputs). Cell IDs stay global: a shard maps its
local indices back through the window it was cut with.
"""
from __future__ import annotations

import torch

from . import amriso


def slab_bounds(x: torch.Tensor, w: torch.Tensor, n_slabs: int, balance: str = "count"):
    """Slab edges [x0, x1) over the cells' x extent: equal widths, or with
    balance="count" (almost) equal numbers of owners per slab."""
    lo, hi = int(x.min()), int((x + w).max())
    if balance == "count":
        xs = torch.sort(x).values
        cuts = [int(xs[k * x.shape[0] // n_slabs]) for k in range(1, n_slabs)]
    else:
        cuts = [lo + (hi - lo) * k // n_slabs for k in range(1, n_slabs)]
    edges = [lo] + cuts + [hi]
    return [(edges[k], edges[k + 1]) for k in range(n_slabs)]


def slab_window(x: torch.Tensor, w: torch.Tensor, x0: int, x1: int, wmax: int) -> torch.Tensor:
    """Indices (increasing) of the cells overlapping [x0 - wmax, x1 + wmax)."""
    return torch.nonzero((x < x1 + wmax) & (x + w > x0 - wmax)).squeeze(1)


def extract_slab(xyz, level, scalar, iso, x0, x1, wmax, device=None, want_duals=True):
    """One shard on the current GPU: its window's cells uploaded, the duals
    owned in [x0, x1) and their triangles at `iso`. Returns (duals int64
    [D, 8] as global cell IDs or None, triangles fp32 [T, 3, 3])."""
    x = xyz[:, 0]
    w = torch.ones_like(x) << level.to(x.dtype)
    win = slab_window(x, w, x0, x1, wmax)
    ctx = amriso.AmrContext(device if device is not None else torch.cuda.current_device())
    try:
        ctx.upload(xyz[win].contiguous(), level[win].contiguous(), scalar[win].contiguous(), copy=True)
        ctx.build_locator()
        ctx.dual_cells(owned_x=(x0, x1))
        duals = win[ctx.get_duals().long()] if want_duals else None
        tris = ctx.iso(iso)
        return duals, tris
    finally:
        ctx.close()


def run_sharded(xyz, level, scalar, iso, n_slabs, rank=0, world=1, group=None, extract=extract_slab,
                want_duals=True):
    """Slab k of n_slabs goes to rank k % world; each rank extracts its slabs
    on its own GPU (the whole cell list is on every rank; each selects its
    windows). Returns this rank's (slab index, duals, triangles) list and the
    per-slab (dual count, triangle count) of all ranks: the one collective is
    the sum of those counts (torch.distributed, when world > 1)."""
    x = xyz[:, 0]
    w = torch.ones_like(x) << level.to(x.dtype)
    wmax = int(w.max())
    bounds = slab_bounds(x, w, n_slabs)
    mine = []
    counts = torch.zeros((n_slabs, 2), dtype=torch.int64)
    for k in range(rank, n_slabs, world):
        x0, x1 = bounds[k]
        d, t = extract(xyz, level, scalar, iso, x0, x1, wmax, want_duals=want_duals)
        mine.append((k, d, t))
        counts[k, 0] = -1 if d is None else d.shape[0]
        counts[k, 1] = t.shape[0]
    if world > 1:
        import torch.distributed as dist
        if dist.get_backend(group) == "nccl":
            c = counts.cuda()
            dist.all_reduce(c, group=group)
            counts = c.cpu()
        else:
            dist.all_reduce(counts, group=group)
    return mine, counts
