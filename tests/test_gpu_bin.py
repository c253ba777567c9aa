"""Before the build: tile binning of an unordered stream (wt_bin) and the
per-pixel depth bounds of §2.1 step 1 (wt_depth_bounds, wt_normalize_depth),
against the oracle's definitions, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import paper_2201_00094_gb300 as wt
import synth
from wtcheck import desc_of

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


def _shuffled(fr: synth.Frame, seed: int):
    """The frame's fragments in a seeded random order (host arrays)."""
    h = fr.numpy()
    perm = np.random.default_rng(seed).permutation(fr.n)
    return {k: h[k][perm] for k in ("pixel", "z", "alpha", "r", "g", "b")}


def _to_dev(h):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to(DEV) for k, v in h.items()}


@pytest.mark.parametrize("tile", [(7, 3), (256, 1), (16, 16)])
def test_bin_groups_an_unordered_stream(tile):
    fr = synth.uniform_frame(53, 37, 5.0, 40, J=3, seed=40 + tile[0], tile_w=tile[0], tile_h=tile[1])
    h = _shuffled(fr, 1)
    d = desc_of(fr)
    g = _to_dev(h)
    out = wt.wt_bin(d, g["pixel"], g["z"], g["alpha"], g["r"], g["g"], g["b"])
    assert wt.wt_get_error() == 0
    order, off = oracle.bin_by_tile(h["pixel"], fr.width, fr.height, *tile)
    got = {k: v.cpu().numpy() for k, v in out.items()}
    np.testing.assert_array_equal(got["tile_offsets"], off)
    # the sort is stable: each tile's fragments in their input order, bit for bit
    for k in ("pixel", "z", "alpha", "r", "g", "b"):
        np.testing.assert_array_equal(got[k][:off[-1]], h[k][order])


@pytest.mark.parametrize("W,H,lam", [(12, 20, 30.0), (300, 200, 1.5), (1500, 1500, 1.5), (4100, 4100, 0.05)])
def test_bin_one_pixel_tiles(W, H, lam):
    """One-pixel tiles: 240 tiles (one radix pass of 8 bits), 60,000 (two),
    2.25M (three) and 16.8M (four passes)."""
    fr = synth.uniform_frame(W, H, lam, 64, J=2, seed=77, tile_w=1, tile_h=1)
    h = _shuffled(fr, 5)
    d = desc_of(fr)
    g = _to_dev(h)
    out = wt.wt_bin(d, g["pixel"], g["z"], g["alpha"], g["r"], g["g"], g["b"])
    assert wt.wt_get_error() == 0
    order, off = oracle.bin_by_tile(h["pixel"], fr.width, fr.height, 1, 1)
    got = {k: v.cpu().numpy() for k, v in out.items()}
    np.testing.assert_array_equal(got["tile_offsets"], off)
    # one tile per pixel: every kept fragment sits in its own pixel's range
    t = np.repeat(np.arange(len(off) - 1), np.diff(off))
    np.testing.assert_array_equal(got["pixel"][: off[-1]], t)
    for k in ("pixel", "z", "alpha", "r", "g", "b"):
        np.testing.assert_array_equal(got[k][:off[-1]], h[k][order])


@pytest.mark.parametrize("n", [1, 31, 8191, 8192, 8193, 3 * 8192 + 5])
def test_bin_ragged_block_edges(n):
    """Stream lengths at and around the sorting block (8192 fragments) and one
    vector (16 keys per thread), over 300 x 7 pixels in 16 x 1 tiles (133
    tiles, one pass) and 1 x 1 tiles (2100 tiles, two passes): the binned
    stream equals the oracle's stable grouping bit for bit."""
    rng = np.random.default_rng(n)
    W, H = 300, 7
    h = {"pixel": rng.integers(0, W * H, n).astype(np.uint32)}
    for k in ("z", "alpha", "r", "g", "b"):
        h[k] = rng.random(n).astype(np.float32)
    g = _to_dev(h)
    for tw, th in ((16, 1), (1, 1)):
        d = wt.make_desc(W, H, 3, tile_w=tw, tile_h=th)
        out = wt.wt_bin(d, g["pixel"], g["z"], g["alpha"], g["r"], g["g"], g["b"])
        assert wt.wt_get_error() == 0
        order, off = oracle.bin_by_tile(h["pixel"], W, H, tw, th)
        got = {k: v.cpu().numpy() for k, v in out.items()}
        np.testing.assert_array_equal(got["tile_offsets"], off)
        for k in ("pixel", "z", "alpha", "r", "g", "b"):
            np.testing.assert_array_equal(got[k][:off[-1]], h[k][order])


def test_binned_stream_composites_like_the_oracle():
    fr = synth.uniform_frame(611, 23, 6.0, 40, J=5, seed=611, tile_w=256, tile_h=1)
    h = _shuffled(fr, 2)
    d = desc_of(fr)
    g = _to_dev(h)
    out = wt.wt_bin(d, g["pixel"], g["z"], g["alpha"], g["r"], g["g"], g["b"])
    frags = wt.make_frags(out["pixel"], out["z"], out["alpha"], out["tile_offsets"], out["r"], out["g"],
                          out["b"])
    res = torch.empty(fr.P, 4, device=DEV)
    wt.wt_build_resolve(d, frags, res, bg=fr.bg)
    assert wt.wt_get_error() == 0
    ref = oracle.composite(h["pixel"], h["z"], h["alpha"], (h["r"], h["g"], h["b"]), fr.P, fr.J, bg=fr.bg)
    np.testing.assert_allclose(res.cpu().numpy(), ref, atol=1e-4, rtol=0)


def test_bin_drops_and_counts_pixels_outside_the_image():
    fr = synth.uniform_frame(40, 24, 4.0, 16, J=3, seed=9)
    h = _shuffled(fr, 3)
    bad = np.array([5, 77, 301])
    h["pixel"] = h["pixel"].copy()
    h["pixel"][bad] = fr.P + np.array([0, 1, 1000])
    d = desc_of(fr)
    g = _to_dev(h)
    out = wt.wt_bin(d, g["pixel"], g["z"], g["alpha"], g["r"], g["g"], g["b"])
    assert wt.wt_get_error() == len(bad)
    off = out["tile_offsets"].cpu().numpy()
    assert off[-1] == fr.n - len(bad)
    _, ref_off = oracle.bin_by_tile(h["pixel"], fr.width, fr.height, fr.tile_w, fr.tile_h)
    np.testing.assert_array_equal(off, ref_off)


def test_bin_empty_stream_and_no_colour():
    d = wt.make_desc(33, 17, 3, tile_w=8, tile_h=4)
    e = torch.empty(0, device=DEV)
    out = wt.wt_bin(d, torch.empty(0, dtype=torch.int32, device=DEV), e, e)
    assert wt.wt_get_error() == 0
    assert out["tile_offsets"].numel() == wt.wt_num_tiles(d) + 1
    assert int(out["tile_offsets"].abs().sum()) == 0
    fr = synth.uniform_frame(33, 17, 3.0, 10, J=3, seed=4, tile_w=8, tile_h=4)
    h = _shuffled(fr, 4)
    g = _to_dev(h)
    out = wt.wt_bin(d, g["pixel"], g["z"], g["alpha"])  # build-only stream: no colour
    _, ref_off = oracle.bin_by_tile(h["pixel"], 33, 17, 8, 4)
    np.testing.assert_array_equal(out["tile_offsets"].cpu().numpy(), ref_off)


def _raw_depth_frame(seed, tile=(16, 16)):
    """A frame whose depths are arbitrary per-pixel affine maps (some negative)
    of depths in [0, 1)."""
    fr = synth.uniform_frame(48, 40, 8.0, 40, J=4, seed=seed, tile_w=tile[0], tile_h=tile[1])
    rng = np.random.default_rng(seed)
    lo_p = rng.uniform(-20, 20, fr.P).astype(np.float32)
    span = rng.uniform(0.01, 50, fr.P).astype(np.float32)
    h = fr.numpy()
    zr = (lo_p[h["pixel"]] + h["z"] * span[h["pixel"]]).astype(np.float32)
    fr.z = torch.from_numpy(zr)
    return fr


def test_depth_bounds_match_the_oracle():
    fr = _raw_depth_frame(21)
    h = fr.numpy()
    g = fr.to(DEV)
    d = desc_of(fr)
    frags = wt.make_frags(g.pixel, g.z, g.alpha, g.tile_offsets, g.r, g.g, g.b)
    zlo = torch.full((fr.P,), float("nan"), device=DEV)
    zhi = torch.full((fr.P,), float("nan"), device=DEV)
    wt.wt_depth_bounds(d, frags, zlo, zhi)
    assert wt.wt_get_error() == 0
    lo, hi = oracle.depth_bounds(h["pixel"], h["z"], h["alpha"], fr.P)
    # min and max of FP32 values are exact
    np.testing.assert_array_equal(zlo.cpu().numpy().astype(np.float64), lo)
    np.testing.assert_array_equal(zhi.cpu().numpy().astype(np.float64), hi)
    assert np.isinf(lo).any()  # some pixels are empty (+inf / -inf)


def test_normalised_depth_and_composite_match_the_oracle():
    fr = _raw_depth_frame(22, tile=(256, 1))
    h = fr.numpy()
    g = fr.to(DEV)
    d = desc_of(fr)
    frags = wt.make_frags(g.pixel, g.z, g.alpha, g.tile_offsets, g.r, g.g, g.b)
    zlo = torch.empty(fr.P, device=DEV)
    zhi = torch.empty(fr.P, device=DEV)
    wt.wt_depth_bounds(d, frags, zlo, zhi)
    zn = torch.empty_like(g.z)
    wt.wt_normalize_depth(d, frags, zlo, zhi, zn)
    lo, hi = oracle.depth_bounds(h["pixel"], h["z"], h["alpha"], fr.P)
    ref_zn = oracle.normalize_depth(h["pixel"], h["z"], fr.P, lo, hi)
    got_zn = zn.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got_zn, ref_zn, atol=4e-7, rtol=0)  # FP32 difference and division
    assert got_zn.min() == 0.0 and got_zn.max() == 1.0
    # the composite on the normalised depths; the oracle gets the same FP32 depths
    frags_n = wt.make_frags(g.pixel, zn, g.alpha, g.tile_offsets, g.r, g.g, g.b)
    out = torch.empty(fr.P, 4, device=DEV)
    wt.wt_build_resolve(d, frags_n, out, bg=fr.bg)
    assert wt.wt_get_error() == 0
    zf = zn.cpu().numpy()
    ref = oracle.composite(h["pixel"], zf, h["alpha"], (h["r"], h["g"], h["b"]), fr.P, fr.J, bg=fr.bg)
    np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-4, rtol=0)
    # in place gives the same depths
    zi = g.z.clone()
    wt.wt_normalize_depth(d, wt.make_frags(g.pixel, zi, g.alpha, g.tile_offsets), zlo, zhi, zi)
    torch.cuda.synchronize()
    assert torch.equal(zi, zn)
    # 16-byte aligned arrays take four fragments per thread, others one: the same
    # depths bit for bit, whatever the count modulo 4
    for cut in (0, 1, 2, 3):
        m = fr.n - cut
        pm = torch.empty(m + 1, dtype=g.pixel.dtype, device=DEV)[1:]
        zm = torch.empty(m + 1, device=DEV)[1:]
        pm.copy_(g.pixel[:m])
        zm.copy_(g.z[:m])
        za = torch.empty(m, device=DEV)
        zb = torch.empty(m + 1, device=DEV)[1:]
        wt.wt_normalize_depth(d, wt.make_frags(g.pixel[:m], g.z[:m], g.alpha, g.tile_offsets), zlo, zhi, za)
        wt.wt_normalize_depth(d, wt.make_frags(pm, zm, g.alpha, g.tile_offsets), zlo, zhi, zb)
        torch.cuda.synchronize()
        assert torch.equal(za, zn[:m]) and torch.equal(zb, zn[:m])


def test_bin_full_size_random_order_frame():
    """The 4K heavy-smoke frame (199M fragments, 192 x 1 tiles) in a seeded
    random order, the preprocessing input of the benchmark: the binned stream
    is the stable sort of that order by tile id (torch's stable sort as the
    reference), the offsets are the frame's own, and two runs agree bit for
    bit."""
    fr = synth.heavy4k(seed=0, device=DEV, tile_w=192, tile_h=1)
    g = torch.Generator(device=DEV)
    g.manual_seed(11)
    perm = torch.randperm(fr.n, device=DEV, generator=g)
    sh = {k: getattr(fr, k)[perm].contiguous() for k in ("pixel", "z", "alpha", "r", "g", "b")}
    del perm
    d = desc_of(fr)
    out = wt.wt_bin(d, sh["pixel"], sh["z"], sh["alpha"], sh["r"], sh["g"], sh["b"])
    assert wt.wt_get_error() == 0
    assert torch.equal(out["tile_offsets"], fr.tile_offsets)
    px = sh["pixel"].long()
    tile = (px // fr.width) * ((fr.width + 191) // 192) + (px % fr.width) // 192
    del px
    order = torch.sort(tile, stable=True).indices
    del tile
    for k in ("pixel", "z", "alpha", "r", "g", "b"):
        assert torch.equal(out[k], sh[k][order]), k
    again = wt.wt_bin(d, sh["pixel"], sh["z"], sh["alpha"], sh["r"], sh["g"], sh["b"])
    assert all(torch.equal(out[k], again[k]) for k in out)
