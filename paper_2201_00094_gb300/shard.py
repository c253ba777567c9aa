"""Splitting one frame across ranks by bands of tile rows.

Pixels are independent (§1.2: a pixel's visibility depends only on its own
fragments, in constant space per pixel), so a frame shards with no exchange
on the data path: rank r builds, resolves and composites the tiles of its own
band with wt_build_resolve_tiles, and the only collective is the optional
gather of the output bands (at most 16 bytes per pixel).

Bands are whole rows of tiles -- contiguous ranges of the row-major tile
order -- so that a band's output is a contiguous range of pixel rows.  They
are balanced by fragment count (the work of the fused kernel grows with the
fragments), read from the stream's tile offsets.  This module is host logic
only; every step of the method runs in the library's kernels.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np
import torch


def tile_grid(desc) -> Tuple[int, int]:
    """(tiles per row, rows of tiles) of a descriptor."""
    ntx = -(-int(desc.width) // int(desc.tile_w))
    nty = -(-int(desc.height) // int(desc.tile_h))
    return ntx, nty


def split_tile_rows(tile_offsets: Sequence[int], desc, world: int) -> List[Tuple[int, int]]:
    """(first_tile, num_tiles) of each rank's band.

    Rank r's band ends at the first boundary between tile rows where the
    running fragment count reaches (r + 1) / world of the frame's fragments
    (rounded to the nearer boundary); every band is a whole number of tile
    rows, the bands are contiguous, in rank order, and cover every tile once.
    A rank may get an empty band when there are fewer tile rows than ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    ntx, nty = tile_grid(desc)
    off = np.asarray(tile_offsets, dtype=np.int64)
    if off.shape[0] < ntx * nty + 1:
        raise ValueError(f"tile_offsets holds {off.shape[0]} entries; the descriptor has {ntx * nty} tiles")
    row_end = off[ntx * np.arange(1, nty + 1)] - off[0]  # fragments up to the end of each tile row
    total = int(row_end[-1]) if nty else 0
    if total == 0:  # no fragments: equal numbers of tile rows
        bounds = [nty * r // world for r in range(world + 1)]
        return [(bounds[r] * ntx, (bounds[r + 1] - bounds[r]) * ntx) for r in range(world)]
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        k = int(np.searchsorted(row_end, target))  # first row whose end reaches the target
        if k > 0 and k < nty and abs(row_end[k - 1] - target) <= abs(row_end[k] - target):
            k -= 1
        rows = min(max(k + 1, bounds[-1]), nty)
        bounds.append(rows)
    bounds.append(nty)
    return [(bounds[r] * ntx, (bounds[r + 1] - bounds[r]) * ntx) for r in range(world)]


def band_rows(rng: Tuple[int, int], desc) -> Tuple[int, int]:
    """The pixel rows [y0, y1) that a band of tiles covers."""
    ntx, _ = tile_grid(desc)
    first, num = rng
    th = int(desc.tile_h)
    y0 = (first // ntx) * th
    y1 = min(((first + num) // ntx) * th, int(desc.height))
    return y0, max(y0, y1)


def build_resolve_band(desc, frags, rng: Tuple[int, int], out: torch.Tensor, coeff=None, zmin=None,
                       bg=(0.5, 0.5, 0.5), bg_img=None, stream=None) -> None:
    """This rank's part of the frame: wt_build_resolve_tiles over its band.
    `out` (and coeff / zmin when given) are full-frame buffers; only the
    band's pixels are written."""
    from . import wt_build_resolve_tiles

    first, num = rng
    if num:
        wt_build_resolve_tiles(desc, frags, first, num, out, coeff, zmin, bg, bg_img, stream)


def gather_bands(out: torch.Tensor, ranges: Sequence[Tuple[int, int]], desc, rank: int,
                 group=None) -> torch.Tensor:
    """All-gathers every rank's band of `out` ([P, 4], the rank's own band
    filled in) into a full frame on every rank.  Bands are padded to the
    largest band for the collective (NCCL for CUDA tensors, gloo for host
    tensors); returns the assembled [P, 4] frame."""
    import torch.distributed as dist

    W = int(desc.width)
    rows = [band_rows(r, desc) for r in ranges]
    longest = max(y1 - y0 for y0, y1 in rows) * W
    y0, y1 = rows[rank]
    mine = torch.zeros(max(longest, 1), out.shape[1], dtype=out.dtype, device=out.device)
    mine[:(y1 - y0) * W] = out[y0 * W:y1 * W]
    parts = [torch.empty_like(mine) for _ in ranges]
    dist.all_gather(parts, mine, group=group)
    frame = torch.empty_like(out)
    for (a, b), part in zip(rows, parts):
        frame[a * W:b * W] = part[:(b - a) * W]
    return frame
