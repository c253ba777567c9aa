"""Seeded synthetic fragment streams shared by the tests, the smoke check and
the benchmark.

This module only draws random inputs.  It holds none of the method's
arithmetic: no clamping, no absorbance, no wavelet maths.  Both the CUDA path
and the CPU oracle consume what it produces.

A frame is a stream of transparent fragments that a rasteriser would produce
for one image (paper §2.1, step 2/3 input): per fragment a pixel id
(y * width + x), a normalised depth z in [0, 1), an opacity alpha and a
surface colour (r, g, b).  The stream is grouped by screen tile (tile_w x
tile_h pixels, tiles in row-major order) with ``tile_offsets[t]`` ..
``tile_offsets[t+1]`` the fragments of tile t, and within a tile the order is
random over pixels and depths, as an unordered raster pass would emit it.

Workloads (the paper's scenes are not available; these stand in for them):

* ``plain64``   64x64, Poisson(4) fragments per pixel capped at 16, z ~ U[0,1),
                alpha ~ U[.05,.6], rgb ~ U[0,1], J = 4.
* ``smoke1080`` 1920x1080; a smoke mask covers exactly 30% of the pixels
                (low-frequency value noise, top 30%); smoke pixels get a
                lognormal count (mean 32, cap 512), depths from three equal
                slabs N(.2/.5/.8, .05) clipped, alpha ~ U[.02,.3]; the other
                pixels get U{0..4} surface fragments, z ~ U[0,1),
                alpha ~ U[.3,.9].  J = 4.
* ``heavy4k``   3840x2160, lognormal count (mean 24, cap 1024); z from a
                5-slab mixture N({.1,.3,.5,.7,.9}, .03) (90%) plus U[0,1)
                (10%), clipped; alpha ~ U[.01,.4].  J = 5.
* ``diff512``   one 512x512 frame of the differentiation batch: Poisson(32)
                capped at 256, z ~ U, alpha ~ U[.05,.5].  J = 4.
* ``serve``     serving frames: resolution drawn from {640x360, 1280x720,
                1920x1080, 3840x2160}, Poisson(lam) counts with lam ~ U[2,32]
                drawn per frame, z ~ U, alpha ~ U[.02,.6].  J = 4.

Lognormal counts use sigma = 1 and mu = ln(mean) - 1/2 so the uncapped mean
is ``mean``; count = min(cap, round(X)).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import torch

TILE = 16
CLIP_HI = 1.0 - 2.0 ** -24  # largest float32 below 1


@dataclasses.dataclass
class Frame:
    width: int
    height: int
    tile_w: int
    tile_h: int
    J: int
    pixel: torch.Tensor         # int32 [n] (pixel ids < 2^31, passed as uint32)
    z: torch.Tensor             # float32 [n]
    alpha: torch.Tensor         # float32 [n]
    r: torch.Tensor             # float32 [n]
    g: torch.Tensor
    b: torch.Tensor
    tile_offsets: torch.Tensor  # int64 [ntiles + 1]
    bg: tuple = (0.5, 0.5, 0.5)
    name: str = ""
    counts: Optional[torch.Tensor] = None  # int32 [P] fragments per pixel

    @property
    def n(self) -> int:
        return int(self.z.numel())

    @property
    def P(self) -> int:
        return self.width * self.height

    @property
    def ntiles(self) -> int:
        return int(self.tile_offsets.numel()) - 1

    def rgb(self) -> torch.Tensor:
        return torch.stack([self.r, self.g, self.b], dim=1)

    def to(self, device) -> "Frame":
        f = dataclasses.replace(self)
        for k in ("pixel", "z", "alpha", "r", "g", "b", "tile_offsets", "counts"):
            v = getattr(self, k)
            if v is not None:
                setattr(f, k, v.to(device))
        return f

    def numpy(self) -> dict:
        return {k: getattr(self, k).cpu().numpy() for k in
                ("pixel", "z", "alpha", "r", "g", "b", "tile_offsets")}


def _gen(device, seed: int) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _uniform(n, lo, hi, g, device):
    return torch.rand(n, generator=g, device=device, dtype=torch.float32) * (hi - lo) + lo


def _lognormal_counts(P, mean, cap, g, device, sigma=1.0):
    mu = math.log(mean) - 0.5 * sigma * sigma
    x = torch.exp(torch.randn(P, generator=g, device=device, dtype=torch.float32) * sigma + mu)
    return torch.clamp(torch.round(x), max=cap).to(torch.int32)


def _poisson_counts(P, lam, cap, g, device):
    rate = torch.full((P,), float(lam), device=device, dtype=torch.float32)
    c = torch.poisson(rate, generator=g).to(torch.int32)
    return torch.clamp(c, max=cap) if cap is not None else c


def assemble(width, height, counts, g, device, tile_w=TILE, tile_h=TILE):
    """Expand per-pixel counts into a tile-grouped, randomly ordered pixel-id
    stream.  Returns (pixel int32 [n], tile_offsets int64 [ntiles+1])."""
    P = width * height
    counts = counts.to(device=device, dtype=torch.int64)
    ntx = (width + tile_w - 1) // tile_w
    nty = (height + tile_h - 1) // tile_h
    ids = torch.arange(P, device=device, dtype=torch.int64)
    tile_of_px = (ids // width // tile_h) * ntx + (ids % width) // tile_w
    tile_counts = torch.zeros(ntx * nty, device=device, dtype=torch.int64)
    tile_counts.index_add_(0, tile_of_px, counts)
    offsets = torch.zeros(ntx * nty + 1, device=device, dtype=torch.int64)
    offsets[1:] = torch.cumsum(tile_counts, 0)
    n = int(offsets[-1].item())
    if n == 0:
        return torch.zeros(0, device=device, dtype=torch.int32), offsets
    pix = torch.repeat_interleave(ids, counts)
    key = tile_of_px[pix] * (1 << 31) + torch.randint(
        0, 1 << 31, (n,), generator=g, device=device, dtype=torch.int64)
    order = torch.sort(key).indices
    del key
    pixel = pix[order].to(torch.int32)
    return pixel, offsets


def _finish(name, width, height, J, pixel, offsets, z, alpha, g, device, counts, tile_w, tile_h):
    n = pixel.numel()
    r = torch.rand(n, generator=g, device=device, dtype=torch.float32)
    gg = torch.rand(n, generator=g, device=device, dtype=torch.float32)
    b = torch.rand(n, generator=g, device=device, dtype=torch.float32)
    return Frame(width, height, tile_w, tile_h, J, pixel, z.contiguous(), alpha.contiguous(), r,
                 gg, b, offsets, (0.5, 0.5, 0.5), name, counts.to(torch.int32))


def uniform_frame(width, height, lam, cap=None, alpha_range=(0.05, 0.6), J=4, seed=0,
                  device="cpu", tile_w=TILE, tile_h=TILE, name="uniform", counts=None):
    """Poisson(lam) fragments per pixel (capped), z ~ U[0,1), alpha ~ U[range]."""
    g = _gen(device, seed)
    P = width * height
    if counts is None:
        counts = _poisson_counts(P, lam, cap, g, device)
    pixel, offsets = assemble(width, height, counts, g, device, tile_w, tile_h)
    n = pixel.numel()
    z = torch.rand(n, generator=g, device=device, dtype=torch.float32)
    alpha = _uniform(n, alpha_range[0], alpha_range[1], g, device)
    return _finish(name, width, height, J, pixel, offsets, z, alpha, g, device, counts,
                   tile_w, tile_h)


def plain64(seed=0, device="cpu", tile_w=TILE, tile_h=TILE):
    return uniform_frame(64, 64, 4.0, 16, (0.05, 0.6), 4, seed, device, tile_w, tile_h,
                         name="plain64")


def _value_noise(width, height, cell, g, device):
    gw = width // cell + 2
    gh = height // cell + 2
    coarse = torch.rand(1, 1, gh, gw, generator=g, device=device, dtype=torch.float32)
    up = torch.nn.functional.interpolate(coarse, size=(gh * cell, gw * cell), mode="bilinear",
                                         align_corners=False)
    return up[0, 0, :height, :width].reshape(-1)


def smoke1080(seed=0, device="cpu", width=1920, height=1080, J=4, tile_w=TILE, tile_h=TILE):
    g = _gen(device, seed)
    P = width * height
    noise = _value_noise(width, height, 64, g, device)
    nsmoke = int(round(0.3 * P))
    smoke = torch.zeros(P, dtype=torch.bool, device=device)
    smoke[torch.argsort(noise, descending=True)[:nsmoke]] = True
    c_smoke = _lognormal_counts(P, 32.0, 512, g, device)
    c_surf = torch.randint(0, 5, (P,), generator=g, device=device, dtype=torch.int32)
    counts = torch.where(smoke, c_smoke, c_surf)
    pixel, offsets = assemble(width, height, counts, g, device, tile_w, tile_h)
    n = pixel.numel()
    is_smoke = smoke[pixel.to(torch.int64)]
    slab = torch.randint(0, 3, (n,), generator=g, device=device)
    means = torch.tensor([0.2, 0.5, 0.8], device=device)[slab]
    z_smoke = torch.clamp(means + 0.05 * torch.randn(n, generator=g, device=device), 0.0, CLIP_HI)
    z_surf = torch.rand(n, generator=g, device=device, dtype=torch.float32)
    z = torch.where(is_smoke, z_smoke, z_surf).to(torch.float32)
    a_smoke = _uniform(n, 0.02, 0.3, g, device)
    a_surf = _uniform(n, 0.3, 0.9, g, device)
    alpha = torch.where(is_smoke, a_smoke, a_surf)
    return _finish("smoke1080", width, height, J, pixel, offsets, z, alpha, g, device, counts,
                   tile_w, tile_h)


def heavy4k(seed=0, device="cpu", width=3840, height=2160, J=5, mean=24.0, cap=1024,
            tile_w=TILE, tile_h=TILE):
    g = _gen(device, seed)
    P = width * height
    counts = _lognormal_counts(P, mean, cap, g, device)
    pixel, offsets = assemble(width, height, counts, g, device, tile_w, tile_h)
    n = pixel.numel()
    slab = torch.randint(0, 5, (n,), generator=g, device=device)
    means = torch.tensor([0.1, 0.3, 0.5, 0.7, 0.9], device=device)[slab]
    z_slab = means + 0.03 * torch.randn(n, generator=g, device=device)
    z_uni = torch.rand(n, generator=g, device=device, dtype=torch.float32)
    pick_uni = torch.rand(n, generator=g, device=device) < 0.1
    z = torch.clamp(torch.where(pick_uni, z_uni, z_slab), 0.0, CLIP_HI).to(torch.float32)
    del z_slab, z_uni, pick_uni, means, slab
    alpha = _uniform(n, 0.01, 0.4, g, device)
    return _finish("heavy4k", width, height, J, pixel, offsets, z, alpha, g, device, counts,
                   tile_w, tile_h)


def diff512(seed=0, device="cpu", width=512, height=512, J=4):
    return uniform_frame(width, height, 32.0, 256, (0.05, 0.5), J, seed, device, name="diff512")


SERVE_SIZES = ((640, 360), (1280, 720), (1920, 1080), (3840, 2160))


def serve_request_params(num, seed=0, mean_gap_ms=2.0):
    """Arrival times (ms), resolution and lambda for ``num`` serving requests."""
    g = _gen("cpu", seed)
    gaps = -torch.log1p(-torch.rand(num, generator=g, dtype=torch.float64)) * mean_gap_ms
    arrivals = torch.cumsum(gaps, 0) - gaps[0]
    size_idx = torch.randint(0, len(SERVE_SIZES), (num,), generator=g)
    lam = torch.rand(num, generator=g, dtype=torch.float64) * 30.0 + 2.0
    return [dict(arrival_ms=float(arrivals[i]), width=SERVE_SIZES[int(size_idx[i])][0],
                 height=SERVE_SIZES[int(size_idx[i])][1], lam=float(lam[i]), seed=seed * 100003 + i)
            for i in range(num)]


def serve_frame(width, height, lam, seed, device="cpu", J=4, tile_w=TILE, tile_h=TILE):
    return uniform_frame(width, height, lam, None, (0.02, 0.6), J, seed, device, tile_w, tile_h,
                         name="serve")


WORKLOADS = {"plain64": plain64, "smoke1080": smoke1080, "heavy4k": heavy4k, "diff512": diff512}


def make(name, seed=0, device="cpu", **kw):
    return WORKLOADS[name](seed=seed, device=device, **kw)


def pixel_subset(frame: Frame, pixels: torch.Tensor):
    """Fragments of a set of pixels (for oracle checks on sampled pixels of a
    large frame).  Returns (index into the stream [m], local pixel id [m]) with
    local ids numbering ``pixels`` in the given order."""
    dev = frame.pixel.device
    pixels = pixels.to(dev, torch.int64)
    lut = torch.full((frame.P,), -1, dtype=torch.int64, device=dev)
    lut[pixels] = torch.arange(pixels.numel(), device=dev)
    loc = lut[frame.pixel.to(torch.int64)]
    idx = torch.nonzero(loc >= 0).squeeze(1)
    return idx, loc[idx]
