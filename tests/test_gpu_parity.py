"""CUDA path vs FP64 oracle, element by element, on seeded synthetic frames
sized so the oracle finishes in seconds but spanning many tiles and ragged
edges.  All calls go through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import paper_2201_00094_gb300 as wt
import synth
from wtcheck import (absorbance_tol, coeff_tol, gpu_run, oracle_run, pixel_counts,
                     pixel_step_sums, desc_of, frags_of)

pytestmark = pytest.mark.gpu

ALL_FLAGS = [7, 6, 5, 4, 3, 2, 1, 0]


def test_plain64_fp32_build_and_composite():
    fr = synth.plain64(seed=0)
    g = gpu_run(fr)
    r = oracle_run(fr)
    assert g["bad"] == 0
    assert (np.abs(g["coeff"] - r["coeff"]) <= coeff_tol(fr)).all()
    np.testing.assert_allclose(g["out"], r["out"], atol=1e-4, rtol=0)


@pytest.mark.parametrize("mode", ["fused", "two_step"])
def test_plain64_other_paths(mode):
    fr = synth.plain64(seed=1)
    g = gpu_run(fr, fused=(mode == "fused"), two_step=(mode == "two_step"))
    r = oracle_run(fr)
    np.testing.assert_allclose(g["out"], r["out"], atol=1e-4, rtol=0)
    if mode == "two_step":
        # only ratios R/W are defined; S is exact
        acc, ref = g["accum"], r["accum"]
        has = ref[:, 3] > 0
        np.testing.assert_allclose(acc[has, :3] / acc[has, 3:4], ref[has, :3] / ref[has, 3:4],
                                   atol=1e-5)
        np.testing.assert_allclose(acc[:, 4], ref[:, 4], rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("J", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("tile", [(16, 16), (8, 4), (7, 3), (1, 1), (16, 1)])
def test_ragged_tiles_every_J(J, tile):
    fr = synth.uniform_frame(53, 37, 5.0, 40, J=J, seed=J * 7 + tile[0], tile_w=tile[0],
                             tile_h=tile[1])
    g = gpu_run(fr)
    r = oracle_run(fr)
    assert g["bad"] == 0
    assert (np.abs(g["coeff"] - r["coeff"]) <= coeff_tol(fr)).all()
    np.testing.assert_allclose(g["out"], r["out"], atol=1e-4, rtol=0)
    gf = gpu_run(fr, fused=True)
    np.testing.assert_allclose(gf["out"], r["out"], atol=1e-4, rtol=0)
    gt = gpu_run(fr, totals=True)
    np.testing.assert_allclose(gt["out"], r["out"], atol=1e-4, rtol=0)


def test_build_totals_are_the_pixels_step_sums():
    """wt_build's optional per-pixel totals: S = sum of the clamped steps,
    against the FP64 sums; 0 for pixels without fragments; under WT_ACCUMULATE
    two batches add up to the whole frame's."""
    fr = synth.uniform_frame(61, 29, 9.0, 120, J=4, seed=77)
    g = gpu_run(fr, totals=True)
    S = pixel_step_sums(fr)
    k = pixel_counts(fr)
    assert (np.abs(g["total"] - S) <= 8 * 2.0 ** -24 * (k + 1) * S).all()
    assert (g["total"][k == 0] == 0).all()
    dev = torch.device("cuda")
    gd = fr.to(dev)
    d1, dA = desc_of(fr), desc_of(fr, flags=wt.DEFAULT_FLAGS | wt.ACCUMULATE)
    coeff = torch.empty(fr.P, 16, device=dev)
    total = torch.empty(fr.P, device=dev)
    f = frags_of(gd)
    wt.wt_build(d1, f, coeff, None, total=total)
    wt.wt_build(dA, f, coeff, None, total=total)  # the same batch again: twice the totals
    torch.cuda.synchronize()
    np.testing.assert_allclose(total.cpu().numpy(), 2 * g["total"], rtol=2e-7, atol=0)


@pytest.mark.parametrize("dtype", [wt.F32, wt.BF16, wt.F16, wt.SE16])
@pytest.mark.parametrize("J,tile,flags", [(4, (16, 16), wt.DEFAULT_FLAGS), (5, (192, 1), wt.DEFAULT_FLAGS),
                                          (3, (7, 3), 3), (6, (16, 16), wt.DEFAULT_FLAGS), (5, (256, 1), 4)])
def test_two_pass_with_totals_equals_fused_bit_for_bit(dtype, J, tile, flags):
    """wt_build + wt_resolve_composite with the build's zmin and totals runs
    the fused kernel's arithmetic in two launches: the same composite, bit for
    bit."""
    fr = synth.uniform_frame(203, 41, 14.0, 200, J=J, seed=J * 31 + tile[0] + flags, tile_w=tile[0],
                             tile_h=tile[1])
    gt = gpu_run(fr, dtype=dtype, flags=flags, totals=True)
    gf = gpu_run(fr, dtype=dtype, flags=flags, fused=True)
    assert gt["bad"] == 0 and gf["bad"] == 0
    np.testing.assert_array_equal(gt["out"], gf["out"])
    np.testing.assert_array_equal(gt["coeff"], gf["coeff"])


def test_row_span_tiles():
    """Tiles one row high (256 x 1, the benchmark's shape) need no division."""
    fr = synth.uniform_frame(611, 23, 6.0, 40, J=5, seed=611, tile_w=256, tile_h=1)
    r = oracle_run(fr)
    for fused in (False, True):
        g = gpu_run(fr, fused=fused)
        assert g["bad"] == 0
        np.testing.assert_allclose(g["out"], r["out"], atol=1e-4, rtol=0)


def test_wide_image_general_row_division():
    """At width 30000 with 16-row tiles the 32-bit reciprocal of the width is
    not exact for every in-tile offset, so the 64-bit one is used."""
    w = 30000
    m = -(-(1 << 32) // w)
    assert (16 * w - 1) * (m * w - (1 << 32)) >= 1 << 32
    fr = synth.uniform_frame(w, 20, 0.3, 8, J=3, seed=30000)
    r = oracle_run(fr)
    g = gpu_run(fr, fused=True)
    assert g["bad"] == 0
    np.testing.assert_allclose(g["out"], r["out"], atol=1e-4, rtol=0)


@pytest.mark.parametrize("flags", ALL_FLAGS)
def test_every_reading_flag(flags):
    fr = synth.uniform_frame(40, 24, 8.0, 64, J=4, seed=100 + flags)
    r = oracle_run(fr, flags=flags)
    for kw in (dict(), dict(fused=True), dict(two_step=True), dict(totals=True),
               dict(two_step=True, totals=True)):
        g = gpu_run(fr, flags=flags, **kw)
        np.testing.assert_allclose(g["out"], r["out"], atol=1e-4, rtol=0, err_msg=str(kw))


def test_zmin_is_nearest_opaque_depth():
    fr = synth.uniform_frame(33, 17, 4.0, 16, J=3, seed=5)
    h = fr.numpy()
    h["alpha"][::5] = 0.0  # transparent fragments do not count
    fr.alpha = torch.from_numpy(h["alpha"])
    g = gpu_run(fr)
    ref = np.full(fr.P, np.inf, np.float32)
    keep = h["alpha"] > 0
    np.minimum.at(ref, h["pixel"][keep].astype(np.int64), np.clip(h["z"][keep], 0, 1 - 2 ** -24))
    np.testing.assert_array_equal(g["zmin"], ref)


@pytest.mark.parametrize("J", [3, 4, 5])
def test_absorbance_queries_match_oracle(J):
    fr = synth.uniform_frame(48, 32, 12.0, 64, J=J, seed=J)
    dev = torch.device("cuda")
    gfr = fr.to(dev)
    d = desc_of(fr)
    coeff = torch.empty(fr.P, 1 << J, device=dev)
    wt.wt_build(d, frags_of(gfr), coeff)
    # fragments themselves (self excluded) and free depth queries
    A = torch.empty(fr.n, device=dev)
    wt.wt_absorbance(d, coeff, gfr.pixel, gfr.z, A, alpha=gfr.alpha)
    rng = np.random.default_rng(J)
    qp = rng.integers(0, fr.P, 5000).astype(np.int32)
    qz = rng.random(5000).astype(np.float32)
    qz[:64] = np.arange(64) / 64.0  # bin edges and centres
    Aq = torch.empty(5000, device=dev)
    wt.wt_absorbance(d, coeff, torch.from_numpy(qp).to(dev), torch.from_numpy(qz).to(dev), Aq)
    assert wt.wt_get_error() == 0
    h = fr.numpy()
    c = oracle.build_coeffs(h["pixel"], h["z"], h["alpha"], fr.P, J)
    S = pixel_step_sums(fr)
    ref = oracle.fragment_absorbance(h["pixel"], h["z"], h["alpha"], fr.P, J, c)
    err = np.abs(A.cpu().numpy() - ref)
    assert (err <= absorbance_tol(ref, S[h["pixel"].astype(np.int64)], J)).all(), err.max()
    refq = oracle.absorbance_at(qp, qz, fr.P, J, c)
    errq = np.abs(Aq.cpu().numpy() - refq)
    assert (errq <= absorbance_tol(refq, S[qp], J)).all(), errq.max()
    # where the pixel holds <= 16 of absorbance, v is within 1e-5 relative
    small = S[h["pixel"].astype(np.int64)] <= 16
    v_rel = np.abs(np.expm1(-(A.cpu().numpy() - ref)))[small]
    assert v_rel.max() <= 1e-5


def test_empty_frame_and_empty_tiles():
    fr = synth.uniform_frame(40, 40, 0.0, 0, J=4, seed=0)
    assert fr.n == 0
    g = gpu_run(fr, bg=(0.1, 0.2, 0.3))
    assert not g["coeff"].any()
    np.testing.assert_array_equal(g["out"], np.tile([0.1, 0.2, 0.3, 0.0], (fr.P, 1)).astype(np.float32))
    assert np.isinf(g["zmin"]).all()
    gf = gpu_run(fr, fused=True, bg=(0.1, 0.2, 0.3))
    np.testing.assert_array_equal(gf["out"], g["out"])


def test_single_fragment_paper_plane():
    """§1.2: one 25%-opaque plane -> 0.25 c + 0.75 bg for every J."""
    for J in range(1, 6):
        counts = torch.zeros(16 * 16, dtype=torch.int32)
        counts[37] = 1
        fr = synth.uniform_frame(16, 16, 0.0, None, J=J, seed=0, counts=counts)
        fr.z[:] = 0.5
        fr.alpha[:] = 0.25
        g = gpu_run(fr, bg=(0.5, 0.5, 0.5))
        c = np.array([fr.r[0], fr.g[0], fr.b[0]], np.float64)
        np.testing.assert_allclose(g["out"][37, :3], 0.25 * c + 0.75 * 0.5, atol=1e-6)
        assert g["out"][37, 3] == pytest.approx(0.25, abs=1e-6)


def test_background_image():
    fr = synth.uniform_frame(37, 29, 3.0, 10, J=4, seed=9)
    bg_img = np.random.default_rng(0).random((fr.P, 3)).astype(np.float32)
    r = oracle_run(fr, bg_img=bg_img)
    for kw in (dict(), dict(fused=True), dict(two_step=True)):
        g = gpu_run(fr, bg_img=bg_img, **kw)
        np.testing.assert_allclose(g["out"], r["out"], atol=1e-4, rtol=0)


def test_bad_fragments_are_skipped_and_counted():
    fr = synth.uniform_frame(32, 32, 4.0, 16, J=4, seed=3)
    h = fr.numpy()
    bad_idx = np.array([0, 5, 17, 300])
    pix = h["pixel"].copy()
    pix[bad_idx[0]] = fr.P + 5                  # outside the image
    pix[bad_idx[1]] = (pix[bad_idx[1]] + 16) % fr.P  # wrong tile (next tile over)
    z = h["z"].copy()
    z[bad_idx[2]] = np.nan
    al = h["alpha"].copy()
    al[bad_idx[3]] = np.nan
    bad_fr = synth.Frame(**{**fr.__dict__, "pixel": torch.from_numpy(pix),
                            "z": torch.from_numpy(z), "alpha": torch.from_numpy(al)})
    g = gpu_run(bad_fr)
    assert g["bad"] == 8  # wt_build and wt_resolve_composite each skip and count the 4
    keep = np.setdiff1d(np.arange(fr.n), bad_idx)
    rgb = (h["r"][keep], h["g"][keep], h["b"][keep])
    c = oracle.build_coeffs(h["pixel"][keep], h["z"][keep], h["alpha"][keep], fr.P, fr.J)
    ref = oracle.resolve(h["pixel"][keep], h["z"][keep], h["alpha"][keep], rgb, fr.P, fr.J, c)[0]
    np.testing.assert_allclose(g["out"], ref, atol=1e-4)
    gf = gpu_run(bad_fr, fused=True)
    assert gf["bad"] == 4
    np.testing.assert_allclose(gf["out"], ref, atol=1e-4)


def test_corrupt_tile_range_is_skipped_and_counted():
    fr = synth.uniform_frame(32, 32, 4.0, 16, J=4, seed=4)
    off = fr.tile_offsets.clone()
    off[2] = off[3] + 1  # tile 1 gets a decreasing range, tile 2 a range past its start
    g = gpu_run(synth.Frame(**{**fr.__dict__, "tile_offsets": off}))
    assert g["bad"] >= 1
    assert np.isfinite(g["out"]).all()


def test_accumulate_batches_equals_single_build():
    fr = synth.uniform_frame(48, 48, 6.0, 32, J=4, seed=11)
    dev = torch.device("cuda")
    g = fr.to(dev)
    d1 = desc_of(fr)
    dA = desc_of(fr, flags=wt.DEFAULT_FLAGS | wt.ACCUMULATE)
    # split every tile's range in two halves -> two batches with their own offsets
    off = fr.tile_offsets
    mid = (off[:-1] + off[1:]) // 2
    idx1 = torch.cat([torch.arange(int(off[t]), int(mid[t])) for t in range(fr.ntiles)])
    idx2 = torch.cat([torch.arange(int(mid[t]), int(off[t + 1])) for t in range(fr.ntiles)])
    off1 = torch.cat([torch.zeros(1, dtype=torch.int64), torch.cumsum(mid - off[:-1], 0)])
    off2 = torch.cat([torch.zeros(1, dtype=torch.int64), torch.cumsum(off[1:] - mid, 0)])
    parts = []
    for idx, o in ((idx1, off1), (idx2, off2)):
        sub = {k: getattr(fr, k)[idx].contiguous().to(dev) for k in ("pixel", "z", "alpha", "r", "g", "b")}
        parts.append((sub, o.to(dev)))
    coeff = torch.empty(fr.P, 16, device=dev)
    zmin = torch.empty(fr.P, device=dev)
    accum = torch.empty(fr.P, 5, device=dev)
    ref_coeff = torch.empty_like(coeff)
    ref_zmin = torch.empty_like(zmin)
    wt.wt_build(d1, frags_of(g), ref_coeff, ref_zmin)
    for i, (sub, o) in enumerate(parts):
        f = wt.make_frags(sub["pixel"], sub["z"], sub["alpha"], o, sub["r"], sub["g"], sub["b"])
        wt.wt_build(d1 if i == 0 else dA, f, coeff, zmin)
    torch.testing.assert_close(coeff, ref_coeff, atol=2e-6, rtol=1e-5)
    torch.testing.assert_close(zmin, ref_zmin, atol=0, rtol=0)
    for i, (sub, o) in enumerate(parts):
        f = wt.make_frags(sub["pixel"], sub["z"], sub["alpha"], o, sub["r"], sub["g"], sub["b"])
        wt.wt_resolve(d1 if i == 0 else dA, f, coeff, zmin, accum)
    out = torch.empty(fr.P, 4, device=dev)
    wt.wt_composite(d1, accum, out)
    r = oracle_run(fr)
    np.testing.assert_allclose(out.cpu().numpy(), r["out"], atol=1e-4)


def test_build_is_deterministic_and_order_independent():
    """Fixed-point bins: the coefficients of a permuted stream are identical."""
    fr = synth.uniform_frame(48, 40, 24.0, 200, J=5, seed=21)
    g1 = gpu_run(fr)
    perm = torch.cat([int(fr.tile_offsets[t]) + torch.randperm(
        int(fr.tile_offsets[t + 1] - fr.tile_offsets[t]), generator=torch.Generator().manual_seed(t))
        for t in range(fr.ntiles)])
    pf = synth.Frame(**{**fr.__dict__, **{k: getattr(fr, k)[perm].contiguous()
                                           for k in ("pixel", "z", "alpha", "r", "g", "b")}})
    for kw in (dict(), dict(fused=True)):
        g2 = gpu_run(pf, **kw)
        np.testing.assert_array_equal(g1["coeff"], g2["coeff"])
    g3 = gpu_run(pf, fused=True)
    g4 = gpu_run(pf, fused=True)
    np.testing.assert_array_equal(g3["out"], g4["out"])


def test_permutation_invariance_on_gpu():
    fr = synth.uniform_frame(32, 32, 10.0, 64, J=5, seed=12)
    g1 = gpu_run(fr)
    perm = torch.cat([int(fr.tile_offsets[t]) + torch.randperm(
        int(fr.tile_offsets[t + 1] - fr.tile_offsets[t]), generator=torch.Generator().manual_seed(t))
        for t in range(fr.ntiles)])
    pf = synth.Frame(**{**fr.__dict__, **{k: getattr(fr, k)[perm].contiguous()
                                           for k in ("pixel", "z", "alpha", "r", "g", "b")}})
    g2 = gpu_run(pf)
    assert (np.abs(g1["coeff"] - g2["coeff"]) <= coeff_tol(fr)).all()
    np.testing.assert_allclose(g1["out"], g2["out"], atol=2e-5)


@pytest.mark.parametrize("J,lam,alpha_range", [(4, 2.0, (1e-4, 0.02)), (5, 40.0, (1e-3, 6e-3)),
                                               (3, 6.0, (1e-6, 0.3))])
def test_fine_steps_keep_their_precision(J, lam, alpha_range):
    """Steps below 2^-7: pixels whose total step is below 2^-7 too are rebuilt
    with per-pixel scales, the others keep the fixed scale (it rounds a step by
    at most 2^-28); either way the coefficients stay within the derived bound
    and the composite within 1e-4, on every path."""
    fr = synth.uniform_frame(67, 29, lam, 200, alpha_range=alpha_range, J=J, seed=int(lam) + J,
                             tile_w=192, tile_h=1)
    r = oracle_run(fr)
    for kw in (dict(), dict(fused=True), dict(totals=True)):
        g = gpu_run(fr, **kw)
        assert g["bad"] == 0
        assert (np.abs(g["coeff"] - r["coeff"]) <= coeff_tol(fr)).all(), kw
        np.testing.assert_allclose(g["out"], r["out"], atol=1e-4, rtol=0, err_msg=str(kw))


def test_deep_pixel_underflow_safe():
    """900 fragments in one depth bin: the nearest sees A ~ 400, every FP32
    exp(-A) underflows; the offset m_p keeps the normalised colour right."""
    k = 900
    counts = torch.zeros(256, dtype=torch.int32)
    counts[0] = k
    counts[1] = 3
    fr = synth.uniform_frame(16, 16, 0.0, None, J=4, seed=0, counts=counts)
    sel = fr.pixel == 0
    fr.z[sel] = (0.5 + torch.arange(k, dtype=torch.float32) / k / 64)[torch.randperm(k)]
    fr.alpha[sel] = 0.6
    r = oracle_run(fr)
    for kw in (dict(), dict(fused=True), dict(two_step=True)):
        g = gpu_run(fr, **kw)
        np.testing.assert_allclose(g["out"], r["out"], atol=1e-4, err_msg=str(kw))


def test_alpha_and_depth_clamps():
    fr = synth.uniform_frame(16, 16, 6.0, 20, J=4, seed=13)
    n = fr.n
    fr.alpha[: n // 4] = 1.0
    fr.alpha[n // 4: n // 3] = -0.2
    fr.z[n // 2: n // 2 + 20] = -1.0
    fr.z[n // 2 + 20: n // 2 + 40] = 2.0
    r = oracle_run(fr)
    g = gpu_run(fr)
    np.testing.assert_allclose(g["out"], r["out"], atol=1e-4)
    assert (np.abs(g["coeff"] - r["coeff"]) <= coeff_tol(fr) * 4).all()


def test_tile_ranges_equal_the_whole_frame():
    """wt_build_resolve_tiles over consecutive tile ranges writes exactly what
    one wt_build_resolve call writes (tiles are independent)."""
    fr = synth.uniform_frame(611, 23, 6.0, 40, J=5, seed=612, tile_w=192, tile_h=1)
    dev = torch.device("cuda")
    g = fr.to(dev)
    d = desc_of(fr)
    f = frags_of(g)
    C = 1 << d.J
    out_a, out_b = torch.empty(fr.P, 4, device=dev), torch.full((fr.P, 4), float("nan"), device=dev)
    c_a, c_b = torch.empty(fr.P, C, device=dev), torch.full((fr.P, C), float("nan"), device=dev)
    wt.wt_build_resolve(d, f, out_a, c_a, bg=fr.bg)
    nt = wt.wt_num_tiles(d)
    cuts = [0, 5, nt // 2, nt]
    for t0, t1 in zip(cuts[:-1], cuts[1:]):
        wt.wt_build_resolve_tiles(d, f, t0, t1 - t0, out_b, c_b, bg=fr.bg)
    wt.wt_build_resolve_tiles(d, f, nt, 0, out_b, c_b, bg=fr.bg)  # empty range: nothing
    assert wt.wt_get_error() == 0
    assert torch.equal(out_a, out_b) and torch.equal(c_a, c_b)
    with pytest.raises(wt.WtError):
        wt.wt_build_resolve_tiles(d, f, nt - 1, 2, out_b, c_b, bg=fr.bg)
    with pytest.raises(wt.WtError):
        wt.wt_build_resolve_tiles(d, f, -1, 1, out_b, c_b, bg=fr.bg)


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("tile", [(192, 1), (16, 16)])
def test_rank_bands_back_to_back_equal_the_whole_frame(world, tile):
    """The ranks' bands of a frame split by tile rows (paper_2201_00094_gb300.shard),
    run one after the other on one GPU, give the whole-frame call's output and
    coefficients bit for bit: every tile is independent of the others."""
    from paper_2201_00094_gb300 import shard

    fr = synth.uniform_frame(611, 97, 7.0, 64, J=5, seed=97 + world, tile_w=tile[0], tile_h=tile[1])
    dev = torch.device("cuda")
    g = fr.to(dev)
    d = desc_of(fr)
    f = frags_of(g)
    ref = torch.empty(fr.P, 4, device=dev)
    cref = torch.empty(fr.P, 32, device=dev)
    wt.wt_build_resolve(d, f, ref, cref, bg=fr.bg)
    ranges = shard.split_tile_rows(fr.tile_offsets.numpy(), d, world)
    assert sum(n for _, n in ranges) == fr.ntiles
    out = torch.full((fr.P, 4), float("nan"), device=dev)
    coeff = torch.full((fr.P, 32), float("nan"), device=dev)
    for rng in ranges:
        shard.build_resolve_band(d, f, rng, out, coeff, bg=fr.bg)
    assert wt.wt_get_error() == 0
    assert torch.equal(out, ref) and torch.equal(coeff, cref)
