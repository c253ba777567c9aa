"""Splitting one frame across ranks by bands of tile rows (host logic; no GPU):
the bands cover every tile exactly once in whole tile rows, are balanced by
fragments, and the gather of the output bands over gloo ranks reassembles the
frame."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import paper_2201_00094_gb300 as wt
from paper_2201_00094_gb300 import shard


def _offsets(rng, ntiles, mean):
    counts = rng.poisson(mean, ntiles)
    counts[rng.random(ntiles) < 0.1] = 0
    return np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)


@pytest.mark.parametrize("size,tile", [((3840, 2160), (192, 1)), ((333, 197), (16, 16)), ((50, 3), (7, 3)),
                                       ((64, 64), (64, 64))])
@pytest.mark.parametrize("world", [1, 2, 3, 5, 8])
def test_bands_cover_every_tile_once_in_whole_rows(size, tile, world):
    d = wt.make_desc(size[0], size[1], 4, tile_w=tile[0], tile_h=tile[1])
    ntx, nty = shard.tile_grid(d)
    rng = np.random.default_rng(world * 131 + size[0])
    off = _offsets(rng, ntx * nty, 50.0)
    ranges = shard.split_tile_rows(off, d, world)
    assert len(ranges) == world
    nxt = 0
    for first, num in ranges:
        assert first == nxt and num >= 0 and first % ntx == 0 and num % ntx == 0
        nxt = first + num
    assert nxt == ntx * nty
    # bands are contiguous pixel rows and tile the image
    rows = [shard.band_rows(r, d) for r in ranges]
    assert rows[0][0] == 0 and rows[-1][1] == size[1]
    assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
    # balanced: each band's fragments are within one tile row of the ideal share
    row_frag = np.diff(off[::ntx][:nty + 1]) if ntx > 0 else None
    per = [int(off[f + n] - off[f]) for f, n in ranges]
    total = int(off[-1])
    if nty >= world:
        assert max(abs(x - total / world) for x in per) <= 1.5 * row_frag.max() + 1


def test_empty_stream_splits_rows_evenly():
    d = wt.make_desc(100, 40, 4, tile_w=10, tile_h=10)  # 10 x 4 tiles
    ranges = shard.split_tile_rows(np.zeros(41, np.int64), d, 3)
    assert ranges == [(0, 10), (10, 10), (20, 20)]
    with pytest.raises(ValueError):
        shard.split_tile_rows(np.zeros(40, np.int64), d, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        d = wt.make_desc(333, 197, 4, tile_w=16, tile_h=16)
        ntx, nty = shard.tile_grid(d)
        off = _offsets(np.random.default_rng(5), ntx * nty, 30.0)
        ranges = shard.split_tile_rows(off, d, world)
        # this rank's band of a full-frame output, filled with a function of
        # the pixel id; the rest holds garbage that must not leak through
        P = d.width * d.height
        out = torch.full((P, 4), float(-1 - rank))
        y0, y1 = shard.band_rows(ranges[rank], d)
        ids = torch.arange(y0 * d.width, y1 * d.width, dtype=torch.float32)
        out[y0 * d.width:y1 * d.width] = torch.stack([ids, ids + 0.25, ids + 0.5, ids + 0.75], dim=1)
        frame = shard.gather_bands(out, ranges, d, rank)
        q.put((rank, ranges, frame.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gathered_bands_reassemble_the_frame(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted((q.get(timeout=120) for _ in range(world)), key=lambda x: x[0])
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    P = 333 * 197
    ids = np.arange(P, dtype=np.float32)
    want = np.stack([ids, ids + 0.25, ids + 0.5, ids + 0.75], axis=1)
    for rank, ranges, frame in res:
        assert ranges == res[0][1]  # every rank derives the same bands
        np.testing.assert_array_equal(frame, want)
