"""Particle rasterisation into the fragment stream (wt_raster_count,
wt_raster_emit) against the oracle's FP32 definition, and the whole chain
particles -> fragments -> tile binning -> build + resolve against the oracle's
composite.  All calls go through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import paper_2201_00094_gb300 as wt

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


def _particles(n, W, H, seed):
    rng = np.random.default_rng(seed)
    p = {"cx": rng.uniform(-8, W + 8, n), "cy": rng.uniform(-8, H + 8, n),
         "radius": rng.uniform(0.3, 7.0, n), "z": rng.random(n), "alpha": rng.uniform(0.05, 0.6, n),
         "r": rng.random(n), "g": rng.random(n), "b": rng.random(n)}
    p = {k: v.astype(np.float32) for k, v in p.items()}
    # a few degenerate particles: zero and negative radius, NaN centre, off screen
    p["radius"][:3] = [0.0, -1.0, 2.0]
    p["cx"][2] = np.nan
    p["cx"][3], p["cy"][3] = W + 100, 5.0
    return p


def _dev(p):
    return {k: torch.from_numpy(v).to(DEV) for k, v in p.items()}


def test_raster_matches_the_oracle_bit_for_bit():
    W, H = 160, 100
    p = _particles(3000, W, H, 1)
    d = wt.make_desc(W, H, 4)
    g = _dev(p)
    out = wt.wt_raster(d, g["cx"], g["cy"], g["radius"], g["z"], g["alpha"], g["r"], g["g"], g["b"])
    assert wt.wt_get_error() == 0
    ref = oracle.raster_particles(W, H, p["cx"], p["cy"], p["radius"], p["z"], p["alpha"], p["r"], p["g"],
                                  p["b"])
    assert int(out["total"]) == len(ref["pixel"]) > 0
    np.testing.assert_array_equal(out["pixel"].cpu().numpy().astype(np.int64), ref["pixel"])
    for k in ("z", "alpha", "r", "g", "b"):
        np.testing.assert_array_equal(out[k].cpu().numpy(), ref[k])


@pytest.mark.parametrize("n", [4096, 4097, 13000])
def test_raster_scan_across_chunks_matches_the_oracle(n):
    """The counts are scanned in chunks of 4096 particles (a scan per chunk,
    then of the chunk totals): one chunk exactly, one particle beyond it, and
    several chunks give the oracle's stream bit for bit."""
    W, H = 128, 96
    p = _particles(n, W, H, 7 + n)
    p["radius"] = (p["radius"] * 0.3).astype(np.float32)  # small discs: a few pixels each
    p["radius"][:3] = [0.0, -1.0, 2.0]
    d = wt.make_desc(W, H, 4)
    g = _dev(p)
    out = wt.wt_raster(d, g["cx"], g["cy"], g["radius"], g["z"], g["alpha"], g["r"], g["g"], g["b"])
    assert wt.wt_get_error() == 0
    ref = oracle.raster_particles(W, H, p["cx"], p["cy"], p["radius"], p["z"], p["alpha"], p["r"], p["g"],
                                  p["b"])
    assert int(out["total"]) == len(ref["pixel"]) > 0
    np.testing.assert_array_equal(out["pixel"].cpu().numpy().astype(np.int64), ref["pixel"])
    for k in ("z", "alpha", "r", "g", "b"):
        np.testing.assert_array_equal(out[k].cpu().numpy(), ref[k])


def test_raster_capacity_drops_and_counts():
    W, H = 64, 48
    p = _particles(300, W, H, 2)
    d = wt.make_desc(W, H, 4)
    g = _dev(p)
    full = wt.wt_raster(d, g["cx"], g["cy"], g["radius"], g["z"], g["alpha"])
    total = int(full["total"])
    cap = total - 37
    part = wt.wt_raster(d, g["cx"], g["cy"], g["radius"], g["z"], g["alpha"], capacity=cap)
    assert wt.wt_get_error() == total - cap
    assert torch.equal(part["pixel"], full["pixel"][:cap]) and torch.equal(part["alpha"], full["alpha"][:cap])


def test_particles_to_composite_match_the_oracle():
    """particles -> wt_raster -> wt_bin -> wt_build_resolve equals the
    oracle's rasterisation and composite."""
    W, H = 384, 64
    p = _particles(4000, W, H, 3)
    d = wt.make_desc(W, H, 5, tile_w=192, tile_h=1)
    g = _dev(p)
    fr = wt.wt_raster(d, g["cx"], g["cy"], g["radius"], g["z"], g["alpha"], g["r"], g["g"], g["b"])
    binned = wt.wt_bin(d, fr["pixel"], fr["z"], fr["alpha"], fr["r"], fr["g"], fr["b"])
    frags = wt.make_frags(binned["pixel"], binned["z"], binned["alpha"], binned["tile_offsets"], binned["r"],
                          binned["g"], binned["b"])
    out = torch.empty(W * H, 4, device=DEV)
    wt.wt_build_resolve(d, frags, out, bg=(0.5, 0.5, 0.5))
    assert wt.wt_get_error() == 0
    ref = oracle.raster_particles(W, H, p["cx"], p["cy"], p["radius"], p["z"], p["alpha"], p["r"], p["g"],
                                  p["b"])
    comp = oracle.composite(ref["pixel"], ref["z"], ref["alpha"], (ref["r"], ref["g"], ref["b"]), W * H, 5)
    np.testing.assert_allclose(out.cpu().numpy(), comp, atol=1e-4, rtol=0)


def test_raster_no_particles():
    d = wt.make_desc(32, 32, 4)
    e = torch.empty(0, device=DEV)
    out = wt.wt_raster(d, e, e, e, e, e)
    assert int(out["total"]) == 0 and out["pixel"].numel() == 0


def _triangles(n, W, H, seed):
    """Random glass panes: quads (two triangles sharing a diagonal) with a
    tilted depth plane, some slivers, one degenerate and one off-screen."""
    rng = np.random.default_rng(seed)
    x, y, z, al = [], [], [], []
    for q in range(n // 2):
        cx, cy = rng.uniform(-10, W + 10), rng.uniform(-10, H + 10)
        u = rng.normal(0, 12, 2)
        v = rng.normal(0, 12, 2)
        p0 = np.array([cx, cy]) - (u + v) / 2
        pts = [p0, p0 + u, p0 + u + v, p0 + v]
        zz = rng.uniform(0, 1, 4)
        for tri in ((0, 1, 2), (0, 2, 3)):
            for k in tri:
                x.append(pts[k][0])
                y.append(pts[k][1])
                z.append(zz[k])
        a = rng.uniform(0.05, 0.6)
        al += [a, a]
    x, y, z, al = (np.asarray(v, dtype=np.float32) for v in (x, y, z, al))
    x[:3] = [5.0, 9.0, 13.0]  # collinear: no area
    y[:3] = [5.0, 9.0, 13.0]
    x[3:6] += 10 * W  # off screen
    rgb = rng.random((3, len(al))).astype(np.float32)
    return {"x": x, "y": y, "z": z, "alpha": al, "r": rgb[0], "g": rgb[1], "b": rgb[2]}


def test_raster_tri_matches_the_oracle_bit_for_bit():
    W, H = 120, 90
    t = _triangles(600, W, H, 5)
    d = wt.make_desc(W, H, 4)
    g = _dev(t)
    out = wt.wt_raster_tri(d, g["x"], g["y"], g["z"], g["alpha"], g["r"], g["g"], g["b"])
    assert wt.wt_get_error() == 0
    ref = oracle.raster_triangles(W, H, t["x"], t["y"], t["z"], t["alpha"], t["r"], t["g"], t["b"])
    assert int(out["total"]) == len(ref["pixel"]) > 0
    np.testing.assert_array_equal(out["pixel"].cpu().numpy().astype(np.int64), ref["pixel"])
    for k in ("z", "alpha", "r", "g", "b"):
        np.testing.assert_array_equal(out[k].cpu().numpy(), ref[k])


def test_raster_tri_panes_to_composite_match_the_oracle():
    """glass panes -> wt_raster_tri -> wt_bin -> wt_build_resolve equals the
    oracle's rasterisation and composite."""
    W, H = 192, 48
    t = _triangles(300, W, H, 6)
    d = wt.make_desc(W, H, 5, tile_w=192, tile_h=1)
    g = _dev(t)
    fr = wt.wt_raster_tri(d, g["x"], g["y"], g["z"], g["alpha"], g["r"], g["g"], g["b"])
    binned = wt.wt_bin(d, fr["pixel"], fr["z"], fr["alpha"], fr["r"], fr["g"], fr["b"])
    frags = wt.make_frags(binned["pixel"], binned["z"], binned["alpha"], binned["tile_offsets"], binned["r"],
                          binned["g"], binned["b"])
    out = torch.empty(W * H, 4, device=DEV)
    wt.wt_build_resolve(d, frags, out, bg=(0.5, 0.5, 0.5))
    assert wt.wt_get_error() == 0
    ref = oracle.raster_triangles(W, H, t["x"], t["y"], t["z"], t["alpha"], t["r"], t["g"], t["b"])
    comp = oracle.composite(ref["pixel"], ref["z"], ref["alpha"], (ref["r"], ref["g"], ref["b"]), W * H, 5)
    np.testing.assert_allclose(out.cpu().numpy(), comp, atol=1e-4, rtol=0)


def test_raster_tri_capacity_and_arguments():
    W, H = 64, 48
    t = _triangles(40, W, H, 7)
    d = wt.make_desc(W, H, 4)
    g = _dev(t)
    full = wt.wt_raster_tri(d, g["x"], g["y"], g["z"], g["alpha"])
    total = int(full["total"])
    part = wt.wt_raster_tri(d, g["x"], g["y"], g["z"], g["alpha"], capacity=total - 11)
    assert wt.wt_get_error() == 11
    assert torch.equal(part["pixel"], full["pixel"][:total - 11])
    e = torch.empty(0, device=DEV)
    none = wt.wt_raster_tri(d, e, e, e, e)
    assert int(none["total"]) == 0
    with pytest.raises(wt.WtError):
        wt.wt_raster_tri(wt.make_desc(1 << 21, 1, 4), g["x"], g["y"], g["z"], g["alpha"])


def test_raster_tri_full_screen_pane():
    """One pane over the whole image (two triangles sharing the diagonal):
    every pixel gets exactly one fragment, bit for bit the oracle's (long walks
    of the bounding box, and the shared edge)."""
    W, H = 160, 100
    x = np.array([0, W, W, 0, W, 0], dtype=np.float32)
    y = np.array([0, 0, H, 0, H, H], dtype=np.float32)
    z = np.array([0.1, 0.5, 0.9, 0.1, 0.9, 0.4], dtype=np.float32)
    al = np.array([0.3, 0.3], dtype=np.float32)
    d = wt.make_desc(W, H, 4)
    g = {k: torch.from_numpy(v).to(DEV) for k, v in (("x", x), ("y", y), ("z", z), ("alpha", al))}
    out = wt.wt_raster_tri(d, g["x"], g["y"], g["z"], g["alpha"])
    assert wt.wt_get_error() == 0
    px = out["pixel"].cpu().numpy().astype(np.int64)
    assert np.array_equal(np.sort(px), np.arange(W * H))
    ref = oracle.raster_triangles(W, H, x, y, z, al)
    np.testing.assert_array_equal(px, ref["pixel"])
    np.testing.assert_array_equal(out["z"].cpu().numpy(), ref["z"])
