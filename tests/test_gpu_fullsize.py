"""Parity at the benchmark's full sizes and launch configuration, on seeded
sampled pixels that the FP64 oracle computes one by one (tiles are
independent, so a pixel's fragments are an exact sub-problem), plus the
accuracy of the absorbance step over the whole clamped alpha range."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2201_00094_gb300 as wt
import synth
from wtcheck import e5_oracle_composite, e5_words_of

pytestmark = pytest.mark.gpu

DT = {"f32": wt.F32, "bf16": wt.BF16, "f16": wt.F16, "se16": wt.SE16}


def test_absorbance_step_accuracy():
    """a = -ln(1 - alpha) for alpha over [0, 1 - 2^-20]: a lone fragment at
    z = 0 has chi_00 = a exactly, so the stored coefficient is the step."""
    al = np.concatenate([np.linspace(0, 1, 200001, dtype=np.float64),
                         1 - np.logspace(-7, -0.3, 5000), np.logspace(-12, -1, 5000)])
    al = np.unique(al.astype(np.float32))
    n = len(al)
    W = 1024
    H = (n + W - 1) // W
    counts = torch.zeros(W * H, dtype=torch.int32)
    counts[:n] = 1
    fr = synth.uniform_frame(W, H, 0.0, None, J=3, seed=0, counts=counts)
    order = fr.pixel.long()  # one fragment per pixel: write alpha by pixel id
    fr.alpha = torch.from_numpy(np.pad(al, (0, W * H - n)))[order].contiguous()
    fr.z = torch.zeros_like(fr.z)
    dev = torch.device("cuda")
    g = fr.to(dev)
    d = wt.make_desc(W, H, 3)
    coeff = torch.empty(W * H, 8, device=dev)
    wt.wt_build(d, wt.make_frags(g.pixel, g.z, g.alpha, g.tile_offsets), coeff)
    got = coeff[:n, 0].double().cpu().numpy()
    ac = np.minimum(al.astype(np.float64), 1 - 2.0 ** -20)
    ref = -np.log1p(-ac)
    rel = np.abs(got - ref) / np.maximum(ref, 1e-300)
    rel[ref == 0] = np.abs(got[ref == 0])
    assert rel.max() < 6e-7, (rel.max(), al[rel.argmax()])


def _sample_check(fr, J, dtype, flags, fused, npix, seed, pixels=None):
    dev = fr.pixel.device
    d = wt.make_desc(fr.width, fr.height, J, DT[dtype], flags, fr.tile_w, fr.tile_h)
    f = wt.make_frags(fr.pixel, fr.z, fr.alpha, fr.tile_offsets, fr.r, fr.g, fr.b)
    coeff = wt.coeff_buffer(d, dev)
    out = torch.empty(fr.P, 4, device=dev)
    if fused:
        wt.wt_build_resolve(d, f, out, coeff, None, bg=fr.bg)
    else:
        zmin = torch.empty(fr.P, device=dev)
        wt.wt_build(d, f, coeff, zmin)
        wt.wt_resolve_composite(d, f, coeff, zmin, out, bg=fr.bg)
    assert wt.wt_get_error() == 0
    if pixels is None:
        pixels = np.random.default_rng(seed).choice(fr.P, npix, replace=False)
    pix = torch.from_numpy(np.asarray(pixels)).to(dev)
    idx, loc = synth.pixel_subset(fr, pix)
    h = {k: getattr(fr, k)[idx].cpu().numpy() for k in ("z", "alpha", "r", "g", "b")}
    loc = loc.cpu().numpy().astype(np.uint32)
    ref = oracle.composite(loc, h["z"], h["alpha"], (h["r"], h["g"], h["b"]), npix, J,
                           flags=flags, bg=fr.bg)
    got = out[pix].cpu().numpy().astype(np.float64)
    err = np.abs(got - ref).max(axis=1)
    counts = np.bincount(loc.astype(np.int64), minlength=npix)
    ac = np.minimum(h["alpha"].astype(np.float64), 1 - 2.0 ** -20)
    S = np.bincount(loc.astype(np.int64), weights=-np.log1p(-ac), minlength=npix)
    return err, counts, S


@pytest.fixture(scope="module")
def heavy4k():
    """The bench's frame in the bench's launch configuration (192 x 1 tiles,
    the four-blocks-per-SM builds); 16 x 16 tiles are covered at 1080p."""
    fr = synth.heavy4k(seed=0, device="cuda", tile_w=192, tile_h=1)
    yield fr
    del fr
    torch.cuda.empty_cache()


@pytest.mark.parametrize("fused", [True, False])
def test_heavy4k_fp32_sampled_pixels(heavy4k, fused):
    """3840x2160 heavy smoke, J = 5, FP32 storage: composites within 1e-4 of
    the FP64 oracle on 4096 seeded sampled pixels."""
    err, counts, _ = _sample_check(heavy4k, 5, "f32", wt.DEFAULT_FLAGS, fused, 4096, seed=4096)
    assert err.max() <= 1e-4, (err.max(), counts[err.argmax()])


# Fragments-per-pixel count below which BF16 storage holds 2e-3 on these
# frames; deeper pixels exceed it (see _check_16bit).
BF16_HOLDS_BELOW = 32


def _check_16bit(err, counts, S, dtype, J, frame, capsys):
    """16-bit coefficient storage, FP32 accumulation: error against FP64 by
    fragments-per-pixel bucket, reported, and asserted against the 2e-3 target
    wherever the format can hold it.

    * SE16 (shared exponent) and FP16 hold 2e-3 on every sampled pixel.
    * BF16 cannot on deep pixels, by its arithmetic: a stored coefficient is
      off by up to u = 2^-8 of itself (8-bit significand); a bin value is
      chi_00 plus J detail terms, of size at most S_p and S_p/2 (S_p = the
      pixel's total step), so |dA| <= u (1 + J/2) S_p, and weights off by
      factors within e^(+-dA) move the normalised colour (a weighted mean of
      colours in [0, 1]) by at most tanh(dA) <= dA.  That bound passes 2e-3
      once S_p > 0.15; measured, BF16 stays within 2e-3 below 32 fragments per
      pixel, which is asserted, and every pixel is held to the bound."""
    edges = [0, 8, 16, 32, 48, 64, 128, 256, 512, 2048]
    rows = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (counts >= lo) & (counts < hi)
        if m.any():
            rows.append((lo, hi, int(m.sum()), float(err[m].max()), float(np.median(err[m]))))
    with capsys.disabled():
        print(f"\n{dtype} storage, {frame}, max|err| by fragments/pixel "
              f"({100 * np.mean(err <= 2e-3):.2f}% of pixels within 2e-3):")
        for r in rows:
            print(f"  [{r[0]:4d},{r[1]:4d}) n={r[2]:5d} max={r[3]:.2e} median={r[4]:.2e}")
    if dtype in ("se16", "f16"):
        assert err.max() <= 2e-3, (err.max(), counts[err.argmax()])
    else:
        u = 2.0 ** -8
        assert (err <= u * (1 + J / 2) * S + 1e-4).all(), float(np.max(err - u * (1 + J / 2) * S))
        shallow = counts < BF16_HOLDS_BELOW
        assert err[shallow].max() <= 2e-3, (err[shallow].max(), counts[shallow][err[shallow].argmax()])


@pytest.mark.parametrize("dtype", ["bf16", "f16", "se16"])
def test_heavy4k_16bit_storage_error_by_depth(heavy4k, dtype, capsys):
    err, counts, S = _sample_check(heavy4k, 5, dtype, wt.DEFAULT_FLAGS, True, 4096, seed=4097)
    _check_16bit(err, counts, S, dtype, 5, "heavy4k", capsys)


@pytest.fixture(scope="module")
def smoke1080():
    fr = synth.smoke1080(seed=0, device="cuda")
    yield fr
    del fr
    torch.cuda.empty_cache()


def test_smoke1080_sampled_pixels(smoke1080):
    for fused in (True, False):
        err, counts, _ = _sample_check(smoke1080, 4, "f32", wt.DEFAULT_FLAGS, fused, 4096, seed=1080)
        assert err.max() <= 1e-4, (err.max(), counts[err.argmax()])


@pytest.mark.parametrize("dtype", ["bf16", "f16", "se16"])
def test_smoke1080_16bit_storage_error_by_depth(smoke1080, dtype, capsys):
    """The 1920x1080 smoke frame (FP32 vs BF16/FP16 storage), 4096 sampled
    pixels weighted to the smoke: half drawn from pixels with 24 or more
    fragments."""
    fr = smoke1080
    cnt = torch.bincount(fr.pixel.long(), minlength=fr.P).cpu().numpy()
    rng = np.random.default_rng(1081)
    deep = np.nonzero(cnt >= 24)[0]
    pix = np.unique(np.concatenate([rng.choice(fr.P, 2048, replace=False),
                                    rng.choice(deep, 2048, replace=False)]))
    err, counts, S = _sample_check(fr, 4, dtype, wt.DEFAULT_FLAGS, True, len(pix), None, pixels=pix)
    _check_16bit(err, counts, S, dtype, 4, "smoke1080", capsys)


def test_fused_equals_two_pass_full_frame(heavy4k):
    fr = heavy4k
    dev = fr.pixel.device
    d = wt.make_desc(fr.width, fr.height, 5, tile_w=fr.tile_w, tile_h=fr.tile_h)
    f = wt.make_frags(fr.pixel, fr.z, fr.alpha, fr.tile_offsets, fr.r, fr.g, fr.b)
    c1 = torch.empty(fr.P, 32, device=dev)
    c2 = torch.empty(fr.P, 32, device=dev)
    o1 = torch.empty(fr.P, 4, device=dev)
    o2 = torch.empty(fr.P, 4, device=dev)
    wt.wt_build_resolve(d, f, o1, c1, None)
    wt.wt_build(d, f, c2, None)
    wt.wt_resolve_composite(d, f, c2, None, o2)
    torch.cuda.synchronize()
    # the coefficients come from order-independent fixed-point bins: identical;
    # the two-pass resolve sums S with FP32 atomics, so the composite agrees
    # to FP32 rounding
    assert torch.equal(c1, c2)
    assert (o1 - o2).abs().max().item() <= 2e-5
    assert math.isfinite(o1.sum().item())
    # with the build's near bounds and totals the two passes run the fused
    # kernel's arithmetic: the same composite bit for bit, at full size
    zmin = torch.empty(fr.P, device=dev)
    total = torch.empty(fr.P, device=dev)
    o3 = torch.empty(fr.P, 4, device=dev)
    wt.wt_build(d, f, c2, zmin, total=total)
    wt.wt_resolve_composite(d, f, c2, zmin, o3, total=total)
    torch.cuda.synchronize()
    assert wt.wt_get_error() == 0
    assert torch.equal(o1, o3)


def test_heavy4k_coloured_sampled_pixels(heavy4k):
    """Coloured absorbance on the bench's frame (opacities alpha x (1, .8, .6)),
    2048 sampled pixels.  FP32 storage: composites within 1e-4 of the oracle.
    E5B9G9R9: the stored words equal, bit for bit, the oracle's encoding of
    the FP32 call's coefficients, and the composite equals the one computed
    wholly on the oracle side (its own encoding) at 1e-4 wherever the two
    encodings agree, within the one-step bound elsewhere."""
    fr = heavy4k
    dev = fr.pixel.device
    d = wt.make_desc(fr.width, fr.height, 5, tile_w=fr.tile_w, tile_h=fr.tile_h)
    f = wt.make_frags(fr.pixel, fr.z, fr.alpha, fr.tile_offsets, fr.r, fr.g, fr.b)
    ac = [fr.alpha, (fr.alpha * 0.8).contiguous(), (fr.alpha * 0.6).contiguous()]
    rng = np.random.default_rng(4100)
    pix = torch.from_numpy(rng.choice(fr.P, 2048, replace=False)).to(dev)
    idx, loc = synth.pixel_subset(fr, pix)
    h = {k: getattr(fr, k)[idx].cpu().numpy() for k in ("z", "r", "g", "b")}
    h["pixel"] = loc.cpu().numpy().astype(np.uint32)
    al = [a[idx].cpu().numpy() for a in ac]
    out = torch.empty(fr.P, 4, device=dev)
    c32 = torch.empty(3, fr.P, 32, device=dev)
    wt.wt_build_resolve_rgb(d, f, *ac, out, c32, wt.RGB_F32, bg=fr.bg)
    assert wt.wt_get_error() == 0
    ref = oracle.composite_rgb(h["pixel"], h["z"], al, (h["r"], h["g"], h["b"]), 2048, 5, bg=fr.bg)
    assert np.abs(out[pix].cpu().numpy() - ref).max() <= 1e-4
    c32s = [c32[c][pix].cpu().numpy() for c in range(3)]
    del c32
    words = torch.empty(fr.P, 32, device=dev, dtype=torch.int32)
    wt.wt_build_resolve_rgb(d, f, *ac, out, words, wt.RGB_E5B9G9R9, bg=fr.bg)
    assert wt.wt_get_error() == 0
    w = words[pix].cpu().numpy().view(np.uint32)
    assert np.array_equal(w, e5_words_of(c32s, 32))
    got = out[pix].cpu().numpy().astype(np.float64)
    ref, bound, same = e5_oracle_composite(h, al, 2048, 5, fr.bg, w)
    err = np.abs(got - ref).max(axis=1)
    assert same.mean() > 0.99
    assert err[same].max() <= 1e-4
    assert (err <= bound).all()


def test_heavy4k_chromatic_aberration_sampled_pixels(heavy4k):
    """wt_composite_ca on the bench's accumulators, background and offset
    field (up to 8 pixels, 5 taps): 4096 sampled pixels against the oracle."""
    fr = heavy4k
    dev = fr.pixel.device
    d = wt.make_desc(fr.width, fr.height, 5, tile_w=fr.tile_w, tile_h=fr.tile_h)
    f = wt.make_frags(fr.pixel, fr.z, fr.alpha, fr.tile_offsets, fr.r, fr.g, fr.b)
    coeff = torch.empty(fr.P, 32, device=dev)
    zmin = torch.empty(fr.P, device=dev)
    acc = torch.empty(fr.P, 5, device=dev)
    wt.wt_build(d, f, coeff, zmin)
    wt.wt_resolve(d, f, coeff, zmin, acc)
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    bg = torch.rand(fr.P, 3, device=dev, generator=g)
    yy = torch.arange(fr.height, device=dev, dtype=torch.float32)[:, None].expand(fr.height, fr.width)
    xx = torch.arange(fr.width, device=dev, dtype=torch.float32)[None, :].expand(fr.height, fr.width)
    off = torch.stack([8.0 * torch.sin(yy / 57.0), 8.0 * torch.cos(xx / 43.0)], dim=-1).reshape(fr.P, 2)
    off = off.contiguous()
    out = torch.empty(fr.P, 4, device=dev)
    wt.wt_composite_ca(d, acc, bg, out, off, 0.5, 5)
    assert wt.wt_get_error() == 0
    rng = np.random.default_rng(4101)
    pix_np = np.sort(rng.choice(fr.P, 4096, replace=False))
    pix = torch.from_numpy(pix_np).to(dev)
    idx, loc = synth.pixel_subset(fr, pix)
    h = {k: getattr(fr, k)[idx].cpu().numpy() for k in ("z", "alpha", "r", "g", "b")}
    loc = loc.cpu().numpy().astype(np.uint32)
    co = oracle.build_coeffs(loc, h["z"], h["alpha"], 4096, 5)
    _, acc_ref = oracle.resolve(loc, h["z"], h["alpha"], (h["r"], h["g"], h["b"]), 4096, 5, co)
    ref = oracle.composite_ca(acc_ref, bg.cpu().numpy(), off.cpu().numpy(), fr.width, fr.height, 0.5, 5,
                              pixels=pix_np)
    err = np.abs(out[pix].cpu().numpy() - ref).max()
    assert err <= 1e-4, err
