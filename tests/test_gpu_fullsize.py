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

pytestmark = pytest.mark.gpu

DT = {"f32": wt.F32, "bf16": wt.BF16, "f16": wt.F16}


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


def _sample_check(fr, J, dtype, flags, fused, npix, seed):
    dev = fr.pixel.device
    d = wt.make_desc(fr.width, fr.height, J, DT[dtype], flags)
    f = wt.make_frags(fr.pixel, fr.z, fr.alpha, fr.tile_offsets, fr.r, fr.g, fr.b)
    coeff = torch.empty(fr.P, 1 << J, device=dev, dtype=wt.coeff_torch_dtype(DT[dtype]))
    out = torch.empty(fr.P, 4, device=dev)
    if fused:
        wt.wt_build_resolve(d, f, out, coeff, None, bg=fr.bg)
    else:
        zmin = torch.empty(fr.P, device=dev)
        wt.wt_build(d, f, coeff, zmin)
        wt.wt_resolve_composite(d, f, coeff, zmin, out, bg=fr.bg)
    assert wt.wt_get_error() == 0
    rng = np.random.default_rng(seed)
    pix = torch.from_numpy(rng.choice(fr.P, npix, replace=False)).to(dev)
    idx, loc = synth.pixel_subset(fr, pix)
    h = {k: getattr(fr, k)[idx].cpu().numpy() for k in ("z", "alpha", "r", "g", "b")}
    loc = loc.cpu().numpy().astype(np.uint32)
    ref = oracle.composite(loc, h["z"], h["alpha"], (h["r"], h["g"], h["b"]), npix, J,
                           flags=flags, bg=fr.bg)
    got = out[pix].cpu().numpy().astype(np.float64)
    err = np.abs(got - ref).max(axis=1)
    counts = np.bincount(loc.astype(np.int64), minlength=npix)
    return err, counts


@pytest.fixture(scope="module")
def heavy4k():
    fr = synth.heavy4k(seed=0, device="cuda")
    yield fr
    del fr
    torch.cuda.empty_cache()


@pytest.mark.parametrize("fused", [True, False])
def test_heavy4k_fp32_sampled_pixels(heavy4k, fused):
    """3840x2160 heavy smoke, J = 5, FP32 storage: composites within 1e-4 of
    the FP64 oracle on 4096 seeded sampled pixels."""
    err, counts = _sample_check(heavy4k, 5, "f32", wt.DEFAULT_FLAGS, fused, 4096, seed=4096)
    assert err.max() <= 1e-4, (err.max(), counts[err.argmax()])


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_heavy4k_16bit_storage_error_by_depth(heavy4k, dtype, capsys):
    """16-bit coefficient storage, FP32 accumulation: error against FP64 by
    fragments-per-pixel bucket.  FP16 keeps 2e-3 everywhere in this frame;
    BF16 (8-bit mantissa) keeps it for pixels of up to 48 fragments, and its
    tail is reported, not hidden."""
    err, counts = _sample_check(heavy4k, 5, dtype, wt.DEFAULT_FLAGS, True, 4096, seed=4097)
    edges = [0, 8, 16, 32, 48, 64, 128, 256, 2048]
    rows = []
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (counts >= lo) & (counts < hi)
        if m.any():
            rows.append((lo, hi, int(m.sum()), float(err[m].max()), float(np.median(err[m]))))
    with capsys.disabled():
        print(f"\n{dtype} storage, heavy4k, max|err| by fragments/pixel:")
        for r in rows:
            print(f"  [{r[0]:4d},{r[1]:4d}) n={r[2]:5d} max={r[3]:.2e} median={r[4]:.2e}")
    if dtype == "f16":
        assert err.max() <= 2e-3
    else:
        assert err[counts < 48].max() <= 2e-3


def test_smoke1080_sampled_pixels():
    fr = synth.smoke1080(seed=0, device="cuda")
    for fused in (True, False):
        err, counts = _sample_check(fr, 4, "f32", wt.DEFAULT_FLAGS, fused, 4096, seed=1080)
        assert err.max() <= 1e-4, (err.max(), counts[err.argmax()])


def test_fused_equals_two_pass_full_frame(heavy4k):
    fr = heavy4k
    dev = fr.pixel.device
    d = wt.make_desc(fr.width, fr.height, 5)
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
