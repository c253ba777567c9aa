"""Coloured absorbance (per-channel opacity, one depth) through the C ABI
against the oracle's definition (each channel is the mono method with its own
opacity and colour component), in FP32 and in the paper's E5B9G9R9 storage."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import paper_2201_00094_gb300 as wt
import synth
from wtcheck import coeff_tol, desc_of, e5_oracle_composite, e5_words_of, frags_of

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


def _coloured(fr: synth.Frame, seed: int):
    """Per-channel opacities: the frame's alpha times a seeded factor per channel."""
    rng = np.random.default_rng(seed)
    a = fr.numpy()["alpha"]
    return [np.clip(a * rng.uniform(0.3, 1.2, fr.n), 0, 0.95).astype(np.float32) for _ in range(3)]


def _check_e5(d, g, a, words, out, h, ac, J, bg=(0.5, 0.5, 0.5), flags=None, bg_img=None, bg_t=None):
    """An E5B9G9R9 call's words and composite: the words equal, bit for bit, the
    oracle's encoding of the coefficients the RGB_F32 call stores; the
    composite equals the one computed wholly on the oracle side at 1e-4 where
    the oracle's own words are the GPU's, within the one-step bound elsewhere."""
    C = 1 << J
    P = words.shape[0]
    c32 = torch.empty(3, P, C, device=DEV)
    wt.wt_build_resolve_rgb(d, frags_of(g), *a, torch.empty(P, 4, device=DEV), c32, wt.RGB_F32, bg=bg,
                            bg_img=bg_t)
    assert wt.wt_get_error() == 0
    w = words.cpu().numpy().view(np.uint32)
    assert np.array_equal(w, e5_words_of(list(c32.cpu().numpy()), C))
    ref, bound, same = e5_oracle_composite(h, ac, P, J, bg, w, flags=flags, bg_img=bg_img)
    err = np.abs(out.cpu().numpy().astype(np.float64) - ref).max(axis=1)
    assert same.mean() > 0.99
    assert err[same].max() <= 1e-4
    assert (err <= bound).all()


@pytest.mark.parametrize("J,tile", [(4, (128, 1)), (5, (64, 1)), (3, (7, 3))])
def test_coloured_fp32_matches_the_oracle(J, tile):
    fr = synth.uniform_frame(96, 40, 8.0, 40, J=J, seed=70 + J, tile_w=tile[0], tile_h=tile[1])
    ac = _coloured(fr, J)
    g = fr.to(DEV)
    d = desc_of(fr)
    a = [torch.from_numpy(x).to(DEV) for x in ac]
    C = 1 << J
    out = torch.empty(fr.P, 4, device=DEV)
    coeff = torch.empty(3, fr.P, C, device=DEV)
    wt.wt_build_resolve_rgb(d, frags_of(g), *a, out, coeff, wt.RGB_F32, bg=(0.2, 0.5, 0.8))
    assert wt.wt_get_error() == 0
    h = fr.numpy()
    rgb = (h["r"], h["g"], h["b"])
    ref = oracle.composite_rgb(h["pixel"], h["z"], ac, rgb, fr.P, J, bg=(0.2, 0.5, 0.8))
    np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-4, rtol=0)
    got = coeff.cpu().numpy().astype(np.float64)
    for c in range(3):
        ref_c = oracle.build_coeffs(h["pixel"], h["z"], ac[c], fr.P, J)
        fc = dataclasses.replace(fr, alpha=torch.from_numpy(ac[c]))
        assert (np.abs(got[c] - ref_c) <= coeff_tol(fc)).all()


def test_grey_opacity_equals_the_mono_method():
    """With the same opacity in every channel the coloured call gives the mono
    call's colour, and each channel's coefficients are the mono build's."""
    fr = synth.uniform_frame(96, 40, 8.0, 40, J=4, seed=80, tile_w=128, tile_h=1)
    g = fr.to(DEV)
    d = desc_of(fr)
    out = torch.empty(fr.P, 4, device=DEV)
    coeff = torch.empty(3, fr.P, 16, device=DEV)
    wt.wt_build_resolve_rgb(d, frags_of(g), g.alpha, g.alpha, g.alpha, out, coeff, wt.RGB_F32, bg=fr.bg)
    mono = torch.empty(fr.P, 4, device=DEV)
    mcoeff = torch.empty(fr.P, 16, device=DEV)
    wt.wt_build_resolve(d, frags_of(g), mono, mcoeff, bg=fr.bg)
    assert wt.wt_get_error() == 0
    torch.testing.assert_close(out, mono, atol=2e-6, rtol=0)
    for c in range(3):
        assert torch.equal(coeff[c], mcoeff)


@pytest.mark.parametrize("J,tile", [(2, (128, 1)), (4, (128, 1)), (5, (128, 1)), (5, (64, 1)), (4, (8, 8)),
                                    (2, (16, 4))])
def test_coloured_e5b9g9r9_storage(J, tile):
    """E5B9G9R9 storage.  The words are byte work: they equal, bit for bit, the
    oracle's encoding of the FP32 coefficients that the RGB_F32 call stores
    (the channels' coefficients come from the same integer bins).  The
    composite equals the oracle's, computed wholly on the oracle side, at
    1e-4 wherever the oracle's words are the GPU's."""
    fr = synth.uniform_frame(96, 40, 8.0, 40, J=J, seed=90 + J, tile_w=tile[0], tile_h=tile[1])
    ac = _coloured(fr, 3)
    g = fr.to(DEV)
    d = desc_of(fr, J)
    C = 1 << J
    a = [torch.from_numpy(x).to(DEV) for x in ac]
    out = torch.empty(fr.P, 4, device=DEV)
    words = torch.empty(fr.P, C, device=DEV, dtype=torch.int32)
    wt.wt_build_resolve_rgb(d, frags_of(g), *a, out, words, wt.RGB_E5B9G9R9, bg=fr.bg)
    c32 = torch.empty(3, fr.P, C, device=DEV)
    wt.wt_build_resolve_rgb(d, frags_of(g), *a, torch.empty(fr.P, 4, device=DEV), c32, wt.RGB_F32, bg=fr.bg)
    assert wt.wt_get_error() == 0
    w = words.cpu().numpy().view(np.uint32)
    assert np.array_equal(w, e5_words_of(list(c32.cpu().numpy()), C))
    h = fr.numpy()
    got = out.cpu().numpy().astype(np.float64)
    ref, bound, same = e5_oracle_composite(h, ac, fr.P, J, fr.bg, w)
    err = np.abs(got - ref).max(axis=1)
    assert same.mean() > 0.99
    assert err[same].max() <= 1e-4
    assert (err <= bound).all()


@pytest.mark.parametrize("J,tile", [(1, (64, 1)), (3, (7, 3)), (4, (128, 1)), (5, (192, 1)), (5, (16, 16)),
                                    (5, (64, 1)), (4, (8, 8)), (2, (16, 4))])
def test_coloured_e5b9g9r9_composite_does_not_depend_on_storing_the_words(J, tile):
    """With a word buffer, channels r and g wait in it (16 bits each) and in
    out until the words are formed; without one, in shared memory.  The
    composite is the same bit for bit, on a frame whose width and height are
    not multiples of the tile, with a background image."""
    fr = synth.uniform_frame(203, 37, 7.0, 35, J=J, seed=300 + 7 * J + tile[1], tile_w=tile[0], tile_h=tile[1])
    ac = _coloured(fr, 23 + J)
    g = fr.to(DEV)
    d = desc_of(fr, J)
    a = [torch.from_numpy(x).to(DEV) for x in ac]
    bg_t = torch.from_numpy(np.random.default_rng(J).random((fr.P, 3)).astype(np.float32)).to(DEV)
    o1 = torch.full((fr.P, 4), float("nan"), device=DEV)
    o2 = torch.full((fr.P, 4), float("nan"), device=DEV)
    words = torch.full((fr.P, 1 << J), -1, device=DEV, dtype=torch.int32)
    wt.wt_build_resolve_rgb(d, frags_of(g), *a, o1, words, wt.RGB_E5B9G9R9, bg_img=bg_t)
    wt.wt_build_resolve_rgb(d, frags_of(g), *a, o2, None, wt.RGB_E5B9G9R9, bg_img=bg_t)
    assert wt.wt_get_error() == 0
    assert torch.equal(o1, o2)
    h = fr.numpy()
    _check_e5(d, g, a, words, o1, h, ac, J, bg_img=bg_t.cpu().numpy(), bg_t=bg_t)


def test_coloured_arguments():
    fr = synth.uniform_frame(32, 8, 2.0, 8, J=4, seed=91, tile_w=32, tile_h=1)
    g = fr.to(DEV)
    d = desc_of(fr)
    out = torch.empty(fr.P, 4, device=DEV)
    with pytest.raises(wt.WtError):
        wt.wt_build_resolve_rgb(d, frags_of(g), g.alpha, g.alpha, g.alpha, out, None, 7, bg=fr.bg)
    with pytest.raises(wt.WtError):
        wt.wt_build_resolve_rgb(d, frags_of(g), g.alpha, None, g.alpha, out, None, wt.RGB_F32, bg=fr.bg)


@pytest.mark.parametrize("tile", [(64, 1), (128, 1)])
def test_coloured_e5b9g9r9_nan_opacity(tile):
    """NaN opacities in one channel, E5B9G9R9 storage: counted once each; the
    composite with the word buffer is the one without it bit for bit, and the
    words are the oracle's encoding of the FP32 call's coefficients."""
    fr = synth.uniform_frame(96, 40, 8.0, 40, J=5, seed=96, tile_w=tile[0], tile_h=tile[1])
    ac = _coloured(fr, 7)
    idx = np.random.default_rng(8).choice(fr.n, 25, replace=False)
    ac[2][idx] = np.nan
    g = fr.to(DEV)
    d = desc_of(fr, 5)
    a = [torch.from_numpy(x).to(DEV) for x in ac]
    o1 = torch.full((fr.P, 4), float("nan"), device=DEV)
    o2 = torch.full((fr.P, 4), float("nan"), device=DEV)
    words = torch.full((fr.P, 32), -1, device=DEV, dtype=torch.int32)
    wt.wt_build_resolve_rgb(d, frags_of(g), *a, o1, words, wt.RGB_E5B9G9R9, bg=fr.bg)
    assert wt.wt_get_error() == 25
    wt.wt_build_resolve_rgb(d, frags_of(g), *a, o2, None, wt.RGB_E5B9G9R9, bg=fr.bg)
    assert wt.wt_get_error() == 25
    assert torch.equal(o1, o2)
    c32 = torch.empty(3, fr.P, 32, device=DEV)
    wt.wt_build_resolve_rgb(d, frags_of(g), *a, torch.empty(fr.P, 4, device=DEV), c32, wt.RGB_F32, bg=fr.bg)
    assert wt.wt_get_error() == 25
    assert np.array_equal(words.cpu().numpy().view(np.uint32), e5_words_of(list(c32.cpu().numpy()), 32))


def test_coloured_nan_opacity_leaves_the_fragment_out_of_that_channel_only():
    """A NaN opacity in one channel drops the fragment from that channel's
    build and resolve alone, and is counted once in the error word."""
    fr = synth.uniform_frame(96, 40, 8.0, 40, J=4, seed=95, tile_w=128, tile_h=1)
    ac = _coloured(fr, 5)
    idx = np.random.default_rng(6).choice(fr.n, 25, replace=False)
    ac[1][idx] = np.nan
    g = fr.to(DEV)
    d = desc_of(fr)
    a = [torch.from_numpy(x).to(DEV) for x in ac]
    out = torch.empty(fr.P, 4, device=DEV)
    coeff = torch.empty(3, fr.P, 16, device=DEV)
    wt.wt_build_resolve_rgb(d, frags_of(g), *a, out, coeff, wt.RGB_F32, bg=fr.bg)
    assert wt.wt_get_error() == 25
    h = fr.numpy()
    col = (h["r"], h["g"], h["b"])
    ref = np.zeros((fr.P, 4))
    for c in range(3):
        keep = ~np.isnan(ac[c])
        px, z, al = h["pixel"][keep], h["z"][keep], ac[c][keep]
        co = oracle.build_coeffs(px, z, al, fr.P, 4)
        o = oracle.resolve(px, z, al, (col[c][keep],) * 3, fr.P, 4, co, bg=(fr.bg[c],) * 3)[0]
        ref[:, c] = o[:, 0]
        ref[:, 3] += o[:, 3] / 3.0
        fc = dataclasses.replace(fr, alpha=torch.from_numpy(np.nan_to_num(ac[c])))
        assert (np.abs(coeff[c].cpu().numpy().astype(np.float64) - co) <= coeff_tol(fc)).all()
    np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-4, rtol=0)


@pytest.mark.parametrize("fmt", [0, 1])
def test_coloured_bg_image_and_256_pixel_tiles(fmt):
    """A background image and the largest tile (256 pixels, 16 x 16) at J = 5."""
    fr = synth.uniform_frame(48, 40, 6.0, 30, J=5, seed=97 + fmt, tile_w=16, tile_h=16)
    ac = _coloured(fr, 7)
    g = fr.to(DEV)
    d = desc_of(fr)
    a = [torch.from_numpy(x).to(DEV) for x in ac]
    bg_img = np.random.default_rng(8).random((fr.P, 3)).astype(np.float32)
    out = torch.empty(fr.P, 4, device=DEV)
    coeff = (torch.empty(3, fr.P, 32, device=DEV) if fmt == wt.RGB_F32
             else torch.empty(fr.P, 32, device=DEV, dtype=torch.int32))
    bgt = torch.from_numpy(bg_img).to(DEV)
    wt.wt_build_resolve_rgb(d, frags_of(g), *a, out, coeff, fmt, bg_img=bgt)
    assert wt.wt_get_error() == 0
    h = fr.numpy()
    if fmt == wt.RGB_E5B9G9R9:
        _check_e5(d, g, a, coeff, out, h, ac, 5, bg_img=bg_img, bg_t=bgt)
        return
    ref = np.zeros((fr.P, 4))
    for c in range(3):
        co = oracle.build_coeffs(h["pixel"], h["z"], ac[c], fr.P, 5)
        col = (h["r"], h["g"], h["b"])[c]
        bgc = np.repeat(bg_img[:, c:c + 1], 3, axis=1)
        o = oracle.resolve(h["pixel"], h["z"], ac[c], (col,) * 3, fr.P, 5, co, bg_img=bgc)[0]
        ref[:, c] = o[:, 0]
        ref[:, 3] += o[:, 3] / 3.0
    np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-4, rtol=0)


@pytest.mark.parametrize("fmt", [0, 1])
def test_coloured_empty_stream(fmt):
    """No fragments: the background, zero coverage, zero coefficients (the
    E5B9G9R9 word of three zeros is 0)."""
    W, H = 50, 7
    d = wt.make_desc(W, H, 4, tile_w=32, tile_h=1)
    e = torch.empty(0, device=DEV)
    pix = torch.empty(0, dtype=torch.int32, device=DEV)
    nt = int(wt.wt_num_tiles(d))
    off = torch.zeros(nt + 1, dtype=torch.int64, device=DEV)
    frags = wt.make_frags(pix, e, e, off, e, e, e)
    out = torch.full((W * H, 4), 7.0, device=DEV)
    coeff = (torch.full((3, W * H, 16), 7.0, device=DEV) if fmt == wt.RGB_F32
             else torch.full((W * H, 16), 7, device=DEV, dtype=torch.int32))
    wt.wt_build_resolve_rgb(d, frags, e, e, e, out, coeff, fmt, bg=(0.1, 0.2, 0.3))
    assert wt.wt_get_error() == 0
    torch.testing.assert_close(out, torch.tensor([0.1, 0.2, 0.3, 0.0], device=DEV).expand(W * H, 4),
                               atol=0, rtol=0)
    assert (coeff == 0).all()


@pytest.mark.parametrize("J", [1, 2])
@pytest.mark.parametrize("fmt", [0, 1])
def test_coloured_short_rows(J, fmt):
    """J = 1 (rows of 8 bytes: no staged stores, words written directly) and
    J = 2, in both storage formats, against the oracle."""
    fr = synth.uniform_frame(70, 30, 6.0, 30, J=J, seed=150 + 2 * J + fmt, tile_w=64, tile_h=1)
    ac = _coloured(fr, 11 + J)
    g = fr.to(DEV)
    d = desc_of(fr)
    a = [torch.from_numpy(x).to(DEV) for x in ac]
    C = 1 << J
    out = torch.empty(fr.P, 4, device=DEV)
    coeff = (torch.empty(3, fr.P, C, device=DEV) if fmt == wt.RGB_F32
             else torch.empty(fr.P, C, device=DEV, dtype=torch.int32))
    wt.wt_build_resolve_rgb(d, frags_of(g), *a, out, coeff, fmt, bg=fr.bg)
    assert wt.wt_get_error() == 0
    h = fr.numpy()
    if fmt == wt.RGB_E5B9G9R9:
        _check_e5(d, g, a, coeff, out, h, ac, J, bg=fr.bg)
        return
    for c in range(3):
        ref_c = oracle.build_coeffs(h["pixel"], h["z"], ac[c], fr.P, J)
        fc = dataclasses.replace(fr, alpha=torch.from_numpy(ac[c]))
        assert (np.abs(coeff[c].cpu().numpy().astype(np.float64) - ref_c) <= coeff_tol(fc)).all()
    ref = oracle.composite_rgb(h["pixel"], h["z"], ac, (h["r"], h["g"], h["b"]), fr.P, J, bg=fr.bg)
    np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-4, rtol=0)


@pytest.mark.parametrize("flags", [wt.SELF_EXCLUDE | wt.INTERP_LINEAR, wt.SELF_EXCLUDE | wt.RESOLVE_NORMALIZED,
                                   wt.INTERP_LINEAR | wt.RESOLVE_NORMALIZED])
@pytest.mark.parametrize("fmt,tile", [(0, (128, 1)), (1, (128, 1)), (1, (64, 1))])
def test_coloured_reading_flags(flags, fmt, tile):
    """The literal resolve, the staircase reconstruction and the fragment's own
    step kept, in both storage formats (the kernels built for arbitrary flags)."""
    fr = synth.uniform_frame(96, 24, 6.0, 30, J=4, seed=160 + flags + 10 * fmt, tile_w=tile[0], tile_h=tile[1])
    ac = _coloured(fr, 17)
    g = fr.to(DEV)
    d = desc_of(fr, flags=flags)
    a = [torch.from_numpy(x).to(DEV) for x in ac]
    out = torch.empty(fr.P, 4, device=DEV)
    coeff = (torch.empty(3, fr.P, 16, device=DEV) if fmt == wt.RGB_F32
             else torch.empty(fr.P, 16, device=DEV, dtype=torch.int32))
    wt.wt_build_resolve_rgb(d, frags_of(g), *a, out, coeff, fmt, bg=fr.bg)
    assert wt.wt_get_error() == 0
    h = fr.numpy()
    if fmt == wt.RGB_E5B9G9R9:
        _check_e5(d, g, a, coeff, out, h, ac, 4, bg=fr.bg, flags=flags)
        return
    ref = oracle.composite_rgb(h["pixel"], h["z"], ac, (h["r"], h["g"], h["b"]), fr.P, 4, flags=flags, bg=fr.bg)
    np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-4, rtol=0)
