"""The single-pass variant of §4: frame t resolved against frame t-1's
coefficients while frame t's are built in the same pass, through the C ABI,
against the oracle's resolve with the previous frame's FP64 coefficients."""
import numpy as np
import pytest
import torch

import oracle
import paper_2201_00094_gb300 as wt
import synth
from wtcheck import coeff_tol, desc_of, frags_of

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


def _frame(seed, J, tile, lam=8.0):
    return synth.uniform_frame(96, 40, lam, 40, J=J, seed=seed, tile_w=tile[0], tile_h=tile[1])


@pytest.mark.parametrize("J,tile", [(6, (192, 1)), (5, (192, 1)), (4, (16, 16)), (3, (7, 3))])
def test_static_scene_equals_the_two_pass_method(J, tile):
    """With frame t-1 = frame t the single pass reproduces the fused call, and
    the coefficients it builds are the build's, bit for bit."""
    fr = _frame(31 + J, J, tile)
    g = fr.to(DEV)
    d = desc_of(fr)
    f = frags_of(g)
    C = 1 << J
    prev = torch.empty(fr.P, C, device=DEV)
    zprev = torch.empty(fr.P, device=DEV)
    wt.wt_build(d, f, prev, zprev)
    ref = torch.empty(fr.P, 4, device=DEV)
    wt.wt_build_resolve(d, f, ref, bg=fr.bg)
    out = torch.empty(fr.P, 4, device=DEV)
    nxt = torch.full((fr.P, C), float("nan"), device=DEV)
    znext = torch.full((fr.P,), float("nan"), device=DEV)
    wt.wt_build_resolve_single_pass(d, f, prev, out, nxt, zprev, znext, bg=fr.bg)
    assert wt.wt_get_error() == 0
    torch.testing.assert_close(out, ref, atol=2e-6, rtol=0)
    assert torch.equal(nxt, prev) and torch.equal(znext, zprev)


@pytest.mark.parametrize("dtype", [wt.F32, wt.BF16, wt.SE16])
def test_moving_scene_matches_the_oracle(dtype):
    """Two different frames: the composite of frame t uses frame t-1's
    visibility exactly as the oracle's resolve with frame t-1's coefficients;
    frame t's coefficients match the oracle's build of frame t."""
    a, b = _frame(41, 4, (192, 1)), _frame(42, 4, (192, 1))
    d = desc_of(b, dtype=dtype)
    ga, gb = a.to(DEV), b.to(DEV)
    C = 16
    prev = wt.coeff_buffer(d, DEV)
    zprev = torch.empty(a.P, device=DEV)
    wt.wt_build(d, frags_of(ga), prev, zprev)
    out = torch.empty(b.P, 4, device=DEV)
    nxt = wt.coeff_buffer(d, DEV)
    wt.wt_build_resolve_single_pass(d, frags_of(gb), prev, out, nxt, zprev, bg=b.bg)
    assert wt.wt_get_error() == 0
    ha, hb = a.numpy(), b.numpy()
    ca = oracle.build_coeffs(ha["pixel"], ha["z"], ha["alpha"], a.P, 4)
    if dtype == wt.F32:
        ref = oracle.resolve(hb["pixel"], hb["z"], hb["alpha"], (hb["r"], hb["g"], hb["b"]), b.P, 4, ca,
                             bg=b.bg)[0]
        np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-4, rtol=0)
        cb = oracle.build_coeffs(hb["pixel"], hb["z"], hb["alpha"], b.P, 4)
        assert (np.abs(nxt.cpu().numpy().astype(np.float64) - cb) <= coeff_tol(b)).all()
    elif dtype == wt.SE16:
        # frame t-1's coefficients encoded on the oracle side
        enc = oracle.se16_decode(*oracle.se16_encode(ca.astype(np.float32), 4), 4)
        ref = oracle.resolve(hb["pixel"], hb["z"], hb["alpha"], (hb["r"], hb["g"], hb["b"]), b.P, 4, enc,
                             bg=b.bg)[0]
        np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-4, rtol=0)
        # frame t's stored codes: the oracle's encoding of the FP32 build's coefficients
        c32 = torch.empty(b.P, C, device=DEV)
        wt.wt_build(desc_of(b), frags_of(gb), c32)
        q, e = oracle.se16_encode(c32.cpu().numpy(), 4)
        gq, ge = oracle.se16_split(nxt.cpu().numpy(), b.P, 4)
        assert np.array_equal(gq, q) and np.array_equal(ge, e)
    else:
        # frame t-1's coefficients rounded to BF16 on the oracle side (to FP32,
        # then to nearest even).  The GPU's FP32 sums can round across a BF16
        # tie differently from the FP64 ones in rare last places; pixels whose
        # stored row differs are left out of the comparison and must be rare.
        bits = ca.astype(np.float32).view(np.uint32).astype(np.uint64)
        bf = (((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16).astype(np.uint32).view(np.float32)
        ref = oracle.resolve(hb["pixel"], hb["z"], hb["alpha"], (hb["r"], hb["g"], hb["b"]), b.P, 4,
                             bf.astype(np.float64), bg=b.bg)[0]
        same = (prev.float().cpu().numpy() == bf).all(axis=1)
        assert same.mean() > 0.99
        np.testing.assert_allclose(out.cpu().numpy()[same], ref[same], atol=1e-4, rtol=0)


def test_single_pass_arguments():
    fr = _frame(50, 4, (192, 1))
    g = fr.to(DEV)
    d = desc_of(fr)
    f = frags_of(g)
    buf = torch.zeros(fr.P, 16, device=DEV)
    out = torch.empty(fr.P, 4, device=DEV)
    with pytest.raises(wt.WtError):  # frame t's coefficients over frame t-1's
        wt.wt_build_resolve_single_pass(d, f, buf, out, buf, bg=fr.bg)
    big = torch.zeros(fr.P + 1, 16, device=DEV)  # overlapping views of full size
    with pytest.raises(wt.WtError):
        wt.wt_build_resolve_single_pass(d, f, big[:-1], out, big[1:], bg=fr.bg)
    # previous coefficients of an empty scene: every fragment fully visible
    wt.wt_build_resolve_single_pass(d, f, buf, out, None, bg=fr.bg)
    h = fr.numpy()
    ref = oracle.resolve(h["pixel"], h["z"], h["alpha"], (h["r"], h["g"], h["b"]), fr.P, 4,
                         np.zeros((fr.P, 16)), flags=wt.INTERP_LINEAR | wt.RESOLVE_NORMALIZED, bg=fr.bg)[0]
    np.testing.assert_allclose(out.cpu().numpy(), ref, atol=1e-4, rtol=0)


def test_j6_with_256_pixel_tiles():
    """At J = 6 with 256-pixel tiles the single pass takes the fused kernel's
    shared memory (the resolve against frame t-1 and frame t's bins share one
    region): an unchanged scene gives the fused call's composite."""
    fr = _frame(51, 6, (16, 16))
    g = fr.to(DEV)
    d = desc_of(fr)
    f = frags_of(g)
    prev = torch.empty(fr.P, 64, device=DEV)
    zprev = torch.empty(fr.P, device=DEV)
    wt.wt_build(d, f, prev, zprev)
    ref = torch.empty(fr.P, 4, device=DEV)
    wt.wt_build_resolve(d, f, ref, bg=fr.bg)
    out = torch.empty(fr.P, 4, device=DEV)
    nxt = torch.full((fr.P, 64), float("nan"), device=DEV)
    wt.wt_build_resolve_single_pass(d, f, prev, out, nxt, zprev, bg=fr.bg)
    assert wt.wt_get_error() == 0
    torch.testing.assert_close(out, ref, atol=2e-6, rtol=0)
    assert torch.equal(nxt, prev)
