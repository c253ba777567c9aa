"""The chromatic-aberration composite (wt_composite_ca, §3) through the C ABI
against the oracle: wt_build + wt_resolve give the accumulators, and the
composite over the tap-gathered background is compared with the oracle's
resolve and composite_ca on the same inputs."""
import numpy as np
import pytest
import torch

import oracle
import paper_2201_00094_gb300 as wt
import synth
from wtcheck import desc_of, frags_of

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


def _accum(fr, flags=wt.DEFAULT_FLAGS):
    """GPU accumulators of the frame (wt_build + wt_resolve) and the oracle's."""
    g = fr.to(DEV)
    d = desc_of(fr, flags=flags)
    C = 1 << fr.J
    coeff = torch.empty(fr.P, C, device=DEV)
    zmin = torch.empty(fr.P, device=DEV)
    wt.wt_build(d, frags_of(g), coeff, zmin)
    acc = torch.empty(fr.P, 5, device=DEV)
    wt.wt_resolve(d, frags_of(g), coeff, zmin, acc)
    h = fr.numpy()
    co = oracle.build_coeffs(h["pixel"], h["z"], h["alpha"], fr.P, fr.J)
    return d, acc, h, co


def _offsets(fr, seed, scale):
    rng = np.random.default_rng(seed)
    P = fr.P
    x = np.arange(P) % fr.width
    y = np.arange(P) // fr.width
    # a smooth swirl plus noise, and some offsets that leave the image
    d = np.stack([scale * np.sin(y / 7.0), scale * np.cos(x / 5.0)], axis=1) + rng.normal(0, 0.3, (P, 2))
    d[rng.choice(P, 20, replace=False)] *= 40.0
    return d.astype(np.float32)


@pytest.mark.parametrize("taps,dispersion,flags", [(5, 0.5, wt.DEFAULT_FLAGS), (1, 0.0, wt.DEFAULT_FLAGS),
                                                   (9, 0.8, wt.DEFAULT_FLAGS), (15, 0.3, wt.DEFAULT_FLAGS),
                                                   (5, 0.5, wt.SELF_EXCLUDE | wt.INTERP_LINEAR)])
def test_composite_ca_matches_the_oracle(taps, dispersion, flags):
    fr = synth.uniform_frame(96, 40, 8.0, 40, J=4, seed=120 + taps, tile_w=128, tile_h=1)
    d, acc, h, co = _accum(fr, flags)
    rng = np.random.default_rng(taps)
    bg = rng.random((fr.P, 3)).astype(np.float32)
    off = _offsets(fr, taps, 6.0)
    out = torch.empty(fr.P, 4, device=DEV)
    wt.wt_composite_ca(d, acc, torch.from_numpy(bg).to(DEV), out, torch.from_numpy(off).to(DEV), dispersion, taps)
    assert wt.wt_get_error() == 0
    _, acc_ref = oracle.resolve(h["pixel"], h["z"], h["alpha"], (h["r"], h["g"], h["b"]), fr.P, fr.J, co, flags,
                                bg_img=bg)
    ref = oracle.composite_ca(acc_ref, bg, off, fr.width, fr.height, dispersion, taps, flags)
    np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-4, rtol=0)


def test_composite_ca_zero_offset_equals_wt_composite():
    """Without an offset every tap reads the pixel's own texel exactly."""
    fr = synth.uniform_frame(96, 40, 8.0, 40, J=4, seed=130, tile_w=128, tile_h=1)
    d, acc, h, co = _accum(fr)
    bg = torch.rand(fr.P, 3, device=DEV)
    a = torch.empty(fr.P, 4, device=DEV)
    b = torch.empty(fr.P, 4, device=DEV)
    wt.wt_composite_ca(d, acc, bg, a, None, 0.5, 5)
    wt.wt_composite(d, acc, b, bg_img=bg)
    assert wt.wt_get_error() == 0
    torch.testing.assert_close(a, b, atol=1e-6, rtol=0)


def test_composite_ca_nonfinite_offsets_are_counted():
    fr = synth.uniform_frame(64, 16, 4.0, 20, J=3, seed=131, tile_w=64, tile_h=1)
    d, acc, h, co = _accum(fr)
    bg = np.random.default_rng(3).random((fr.P, 3)).astype(np.float32)
    off = _offsets(fr, 4, 3.0)
    off[5] = [np.nan, 0.0]
    off[9] = [0.0, np.inf]
    off[11] = [-np.inf, np.nan]
    out = torch.empty(fr.P, 4, device=DEV)
    wt.wt_composite_ca(d, acc, torch.from_numpy(bg).to(DEV), out, torch.from_numpy(off).to(DEV), 0.5, 5)
    assert wt.wt_get_error() == 3
    _, acc_ref = oracle.resolve(h["pixel"], h["z"], h["alpha"], (h["r"], h["g"], h["b"]), fr.P, fr.J, co,
                                bg_img=bg)
    ref = oracle.composite_ca(acc_ref, bg, off, fr.width, fr.height, 0.5, 5)
    np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-4, rtol=0)


def test_composite_ca_arguments():
    fr = synth.uniform_frame(32, 8, 2.0, 8, J=3, seed=132, tile_w=32, tile_h=1)
    d, acc, h, co = _accum(fr)
    bg = torch.rand(fr.P, 3, device=DEV)
    out = torch.empty(fr.P, 4, device=DEV)
    for taps, disp in ((0, 0.5), (4, 0.5), (17, 0.5), (5, -1.0), (5, float("nan"))):
        with pytest.raises(wt.WtError):
            wt.wt_composite_ca(d, acc, bg, out, None, disp, taps)
    with pytest.raises(wt.WtError):
        wt.wt_composite_ca(d, acc, None, out, None, 0.5, 5)
    # taller than the launch grid allows (more than 65535 rows of 16-pixel tiles)
    tall = wt.make_desc(1, 1 << 20, 3)
    acc_t = torch.zeros(1 << 20, 5, device=DEV)
    bg_t = torch.zeros(1 << 20, 3, device=DEV)
    out_t = torch.empty(1 << 20, 4, device=DEV)
    with pytest.raises(wt.WtError):
        wt.wt_composite_ca(tall, acc_t, bg_t, out_t, None, 0.5, 5)


@pytest.mark.parametrize("W,H", [(1, 37), (130, 70)])
def test_composite_ca_thin_and_ragged_images(W, H):
    """A one-pixel-wide image (every staged texel clamps to column 0) and an
    image whose tiles are ragged on both sides, with offsets that leave the
    staged halo."""
    fr = synth.uniform_frame(W, H, 3.0, 20, J=3, seed=140 + W, tile_w=1 if W == 1 else 130, tile_h=1)
    d, acc, h, co = _accum(fr)
    rng = np.random.default_rng(W)
    bg = rng.random((fr.P, 3)).astype(np.float32)
    off = rng.normal(0, 9, (fr.P, 2)).astype(np.float32)
    out = torch.empty(fr.P, 4, device=DEV)
    wt.wt_composite_ca(d, acc, torch.from_numpy(bg).to(DEV), out, torch.from_numpy(off).to(DEV), 0.7, 7)
    assert wt.wt_get_error() == 0
    _, acc_ref = oracle.resolve(h["pixel"], h["z"], h["alpha"], (h["r"], h["g"], h["b"]), fr.P, fr.J, co,
                                bg_img=bg)
    ref = oracle.composite_ca(acc_ref, bg, off, fr.width, fr.height, 0.7, 7)
    np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-4, rtol=0)
