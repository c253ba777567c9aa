"""Shared-exponent 16-bit coefficient storage (WT_SE16) against the oracle.

* The stored codes are integer work: the mantissas and exponent bytes of every
  call that stores coefficients are compared bit for bit with the oracle's
  encoder applied to the same FP32 coefficients (those of the FP32-storage
  call, which come from the same order-independent integer bins).
* The composite is compared with an oracle that encodes its own coefficients
  (FP64 closed form, rounded to FP32, encoded and decoded on the oracle side),
  at the FP32 path's 1e-4, and with the unquantised FP64 composite at the
  16-bit storage target, 2e-3."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
import paper_2201_00094_gb300 as wt
import synth
from wtcheck import desc_of, frags_of

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


def _codes(buf, fr, J):
    mant, expo = oracle.se16_split(buf.cpu().numpy(), fr.P, J)
    return mant.copy(), expo.copy()


def _oracle_se16_coeffs(h, P, J):
    c32 = oracle.build_coeffs(h["pixel"], h["z"], h["alpha"], P, J).astype(np.float32)
    q, e = oracle.se16_encode(c32, J)
    return oracle.se16_decode(q, e, J)


@pytest.mark.parametrize("J", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("tile", [(16, 16), (7, 3), (192, 1)])
def test_codes_bit_exact_every_path(J, tile):
    fr = synth.uniform_frame(197, 61, 9.0, 96, J=J, seed=40 + J, tile_w=tile[0], tile_h=tile[1])
    g = fr.to(DEV)
    f = frags_of(g)
    d32 = desc_of(fr, J, wt.F32)
    dse = desc_of(fr, J, wt.SE16)
    c32 = torch.empty(fr.P, 1 << J, device=DEV)
    wt.wt_build(d32, f, c32)
    want_q, want_e = oracle.se16_encode(c32.cpu().numpy(), J)
    out = torch.empty(fr.P, 4, device=DEV)
    bufs = {}
    for name in ("build", "fused", "single_pass"):
        b = torch.full((wt.coeff_storage_bytes(dse),), 0xA5, dtype=torch.uint8, device=DEV)
        if name == "build":
            wt.wt_build(dse, f, b)
        elif name == "fused":
            wt.wt_build_resolve(dse, f, out, b)
        else:
            prev = wt.coeff_buffer(dse, DEV)
            wt.wt_build(dse, f, prev)
            wt.wt_build_resolve_single_pass(dse, f, prev, out, b)
        bufs[name] = b
    assert wt.wt_get_error() == 0
    for name, b in bufs.items():
        q, e = _codes(b, fr, J)
        assert np.array_equal(e, want_e), name
        assert np.array_equal(q, want_q), name


@pytest.mark.parametrize("J", [2, 4, 5])
@pytest.mark.parametrize("fused", [True, False])
def test_composite_vs_oracle_encoding(J, fused):
    fr = synth.uniform_frame(131, 77, 20.0, 400, alpha_range=(0.02, 0.6), J=J, seed=50 + J)
    g = fr.to(DEV)
    f = frags_of(g)
    d = desc_of(fr, J, wt.SE16)
    coeff = wt.coeff_buffer(d, DEV)
    zmin = torch.empty(fr.P, device=DEV)
    out = torch.full((fr.P, 4), float("nan"), device=DEV)
    if fused:
        wt.wt_build_resolve(d, f, out, coeff, zmin, bg=fr.bg)
    else:
        wt.wt_build(d, f, coeff, zmin)
        wt.wt_resolve_composite(d, f, coeff, zmin, out, bg=fr.bg)
    assert wt.wt_get_error() == 0
    h = fr.numpy()
    rgb = (h["r"], h["g"], h["b"])
    ref = oracle.resolve(h["pixel"], h["z"], h["alpha"], rgb, fr.P, J, _oracle_se16_coeffs(h, fr.P, J),
                         bg=fr.bg)[0]
    got = out.cpu().numpy().astype(np.float64)
    assert np.abs(got - ref).max() <= 1e-4
    exact = oracle.composite(h["pixel"], h["z"], h["alpha"], rgb, fr.P, J, bg=fr.bg)
    assert np.abs(got - exact).max() <= 2e-3


@pytest.mark.parametrize("flags", [0, 1, 3, 5, 7])
def test_reading_flags_and_accumulate(flags):
    """Every reading, and a frame built in two batches (WT_ACCUMULATE decodes
    the stored row, adds, and encodes again)."""
    fr = synth.uniform_frame(64, 40, 10.0, 64, J=4, seed=60 + flags)
    g = fr.to(DEV)
    d = desc_of(fr, 4, wt.SE16, flags)
    coeff = wt.coeff_buffer(d, DEV)
    out = torch.empty(fr.P, 4, device=DEV)
    wt.wt_build(d, frags_of(g), coeff)
    wt.wt_resolve_composite(d, frags_of(g), coeff, None, out, bg=fr.bg)
    h = fr.numpy()
    rgb = (h["r"], h["g"], h["b"])
    ref = oracle.resolve(h["pixel"], h["z"], h["alpha"], rgb, fr.P, 4, _oracle_se16_coeffs(h, fr.P, 4),
                         flags=flags, bg=fr.bg)[0]
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-4
    if flags == 7:
        # two batches of every tile (its first half, then the rest), the
        # second added under WT_ACCUMULATE, which decodes the stored row, adds
        # the batch's FP32 coefficients in FP32 and encodes again
        off = g.tile_offsets
        idx = torch.arange(fr.n, device=DEV)
        t = torch.searchsorted(off[1:], idx, right=True)
        first = idx < (off[:-1] + (off[1:] - off[:-1]) // 2)[t]
        parts = []
        for m in (first, ~first):
            sub = dataclasses.replace(fr)
            sel = m.cpu()
            for k in ("pixel", "z", "alpha", "r", "g", "b"):
                setattr(sub, k, getattr(fr, k)[sel].contiguous())
            cnt = torch.bincount(t[m], minlength=fr.ntiles).cpu()
            sub.tile_offsets = torch.cat([torch.zeros(1, dtype=torch.int64), torch.cumsum(cnt, 0)])
            parts.append(sub.to(DEV))
        acc = wt.coeff_buffer(d, DEV)
        wt.wt_build(d, frags_of(parts[0]), acc)
        wt.wt_build(desc_of(fr, 4, wt.SE16, flags | wt.ACCUMULATE), frags_of(parts[1]), acc)
        c32 = []
        for part in parts:  # each batch's FP32 coefficients (the same integer bins)
            c = torch.empty(fr.P, 16, device=DEV)
            wt.wt_build(desc_of(fr, 4, wt.F32, flags), frags_of(part), c)
            c32.append(c.cpu().numpy())
        assert wt.wt_get_error() == 0
        first_dec = oracle.se16_decode(*oracle.se16_encode(c32[0], 4), 4).astype(np.float32)  # exact
        want_q, want_e = oracle.se16_encode(c32[1] + first_dec, 4)
        q, e = _codes(acc, fr, 4)
        assert np.array_equal(e, want_e) and np.array_equal(q, want_q)


def test_absorbance_queries():
    J = 5
    fr = synth.uniform_frame(48, 32, 12.0, 64, J=J, seed=70)
    g = fr.to(DEV)
    d = desc_of(fr, J, wt.SE16)
    coeff = wt.coeff_buffer(d, DEV)
    wt.wt_build(d, frags_of(g), coeff)
    A = torch.empty(fr.n, device=DEV)
    wt.wt_absorbance(d, coeff, g.pixel, g.z, A, g.alpha)
    assert wt.wt_get_error() == 0
    h = fr.numpy()
    dec = oracle.se16_decode(*_codes(coeff, fr, J), J)
    ref = oracle.fragment_absorbance(h["pixel"], h["z"], h["alpha"], fr.P, J, dec)
    tol = 1e-5 * np.maximum(1.0, ref) + 1e-5
    assert (np.abs(A.cpu().numpy() - ref) <= tol).all()


def test_empty_and_transparent_pixels():
    """Pixels without fragments, or with alpha = 0 only, store zero mantissas
    and the smallest exponent, and composite to the background."""
    fr = synth.uniform_frame(40, 30, 3.0, 8, J=4, seed=71)
    h = fr.numpy()
    h["alpha"][h["pixel"] % 3 == 0] = 0.0
    fr.alpha = torch.from_numpy(h["alpha"])
    g = fr.to(DEV)
    d = desc_of(fr, 4, wt.SE16)
    coeff = wt.coeff_buffer(d, DEV)
    out = torch.empty(fr.P, 4, device=DEV)
    wt.wt_build_resolve(d, frags_of(g), out, coeff, bg=(0.25, 0.5, 0.75))
    q, e = _codes(coeff, fr, 4)
    cnt = np.bincount(h["pixel"][h["alpha"] > 0].astype(np.int64), minlength=fr.P)
    empty = cnt == 0
    assert empty.any()
    assert not q[empty].any() and (e[empty] == 28).all()
    np.testing.assert_allclose(out.cpu().numpy()[empty], [[0.25, 0.5, 0.75, 0.0]] * int(empty.sum()),
                               atol=0)
