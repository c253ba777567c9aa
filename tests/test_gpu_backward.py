"""Adjoint of build + resolve + composite on the GPU (wt_backward) against the
FP64 oracle: its analytic gradient (itself pinned to finite differences in
test_oracle.py) on small frames, and FP64 central finite differences of the
oracle's composite on 512 sampled fragments of the differentiation workload
(16 frames of 512x512, Poisson(32) fragments per pixel)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2201_00094_gb300 as wt
import synth

pytestmark = pytest.mark.gpu


def _gpu_grad(fr, gout, J=None, flags=wt.DEFAULT_FLAGS, bg=(0.5, 0.5, 0.5), bg_img=None):
    dev = torch.device("cuda")
    g = fr.to(dev)
    d = wt.make_desc(fr.width, fr.height, fr.J if J is None else J, wt.F32, flags, fr.tile_w,
                     fr.tile_h)
    f = wt.make_frags(g.pixel, g.z, g.alpha, g.tile_offsets, g.r, g.g, g.b)
    ga = torch.full((fr.n,), float("nan"), device=dev)
    gc = torch.full((3, fr.n), float("nan"), device=dev)
    bgt = None if bg_img is None else torch.as_tensor(bg_img, dtype=torch.float32, device=dev)
    wt.wt_backward(d, f, torch.as_tensor(gout, dtype=torch.float32, device=dev).contiguous(), ga,
                   gc, bg=bg, bg_img=bgt)
    assert wt.wt_get_error() == 0
    return ga.double().cpu().numpy(), gc.double().cpu().numpy().T


def _ref_grad(fr, gout, J=None, flags=wt.DEFAULT_FLAGS, bg=(0.5, 0.5, 0.5), bg_img=None):
    h = fr.numpy()
    return oracle.grad(h["pixel"], h["z"], h["alpha"], (h["r"], h["g"], h["b"]), fr.P,
                       fr.J if J is None else J, gout, flags=flags, bg=bg, bg_img=bg_img)


def _close(got, ref, rel=1e-3, absfrac=1e-5):
    tol = rel * np.abs(ref) + absfrac * max(np.abs(ref).max(), 1e-30)
    bad = np.abs(got - ref) > tol
    assert not bad.any(), (np.abs(got - ref).max(), int(bad.sum()), got[bad][:5], ref[bad][:5])


@pytest.mark.parametrize("flags", [7, 3, 5, 6, 4, 1])
@pytest.mark.parametrize("J", [2, 4, 5, 6])
def test_backward_matches_oracle_gradient(flags, J):
    fr = synth.uniform_frame(37, 29, 6.0, 40, alpha_range=(0.05, 0.6), J=J, seed=30 + J + flags)
    gout = np.random.default_rng(J + flags).standard_normal((fr.P, 4))
    ga, gc = _gpu_grad(fr, gout, flags=flags)
    ra, rc = _ref_grad(fr, gout, flags=flags)
    _close(ga, ra)
    _close(gc, rc)


def test_backward_background_image_and_clamped_alpha():
    fr = synth.uniform_frame(33, 21, 8.0, 40, alpha_range=(0.05, 0.6), J=4, seed=77)
    fr.alpha[::17] = 1.0      # clamped: zero gradient
    fr.alpha[5::23] = 0.0     # clamped: zero gradient
    bg_img = np.random.default_rng(1).random((fr.P, 3)).astype(np.float32)
    gout = np.random.default_rng(2).standard_normal((fr.P, 4))
    ga, gc = _gpu_grad(fr, gout, bg_img=bg_img)
    ra, rc = _ref_grad(fr, gout, bg_img=bg_img)
    _close(ga, ra)
    _close(gc, rc)
    assert (ga[::17] == 0).all() and (ga[5::23] == 0).all()


def test_backward_is_the_same_on_every_run():
    """The scatter of gamma into the bins is integer fixed point, so two runs
    on the same inputs give the same gradients bit for bit."""
    fr = synth.uniform_frame(64, 48, 30.0, 200, alpha_range=(0.02, 0.6), J=5, seed=91, tile_w=192,
                             tile_h=1)
    gout = np.random.default_rng(91).standard_normal((fr.P, 4))
    a1, c1 = _gpu_grad(fr, gout)
    a2, c2 = _gpu_grad(fr, gout)
    np.testing.assert_array_equal(a1, a2)
    np.testing.assert_array_equal(c1, c2)
    ra, rc = _ref_grad(fr, gout)
    _close(a1, ra)
    _close(c1, rc)


@pytest.mark.parametrize("flags", [7, 3])
def test_backward_with_colours_beyond_one(flags):
    """Colours far outside [0, 1] break the bound the fixed-point scale of the
    gamma scatter assumes; the tiles where a term or a sum would not fit take
    the FP32 scatter, and the gradients still match the oracle."""
    fr = synth.uniform_frame(40, 30, 12.0, 80, alpha_range=(0.05, 0.6), J=4, seed=55 + flags)
    rng = np.random.default_rng(5)
    for ch in ("r", "g", "b"):
        setattr(fr, ch, torch.from_numpy((rng.random(fr.n) * 4000.0 - 2000.0).astype(np.float32)))
    gout = rng.standard_normal((fr.P, 4))
    ga, gc = _gpu_grad(fr, gout, flags=flags)
    ra, rc = _ref_grad(fr, gout, flags=flags)
    _close(ga, ra)
    _close(gc, rc)


@pytest.mark.parametrize("flags,J,tile", [(7, 4, (16, 16)), (7, 5, (192, 1)), (3, 4, (7, 5)), (5, 5, (16, 16))])
def test_backward_with_the_forward_sums_is_the_same(flags, J, tile):
    """Given the pixel sums wt_build_resolve stored, wt_backward skips
    recomputing them: the gradients are the same, bit for bit."""
    fr = synth.uniform_frame(97, 41, 18.0, 120, alpha_range=(0.02, 0.6), J=J, seed=40 + flags + J,
                             tile_w=tile[0], tile_h=tile[1])
    dev = torch.device("cuda")
    g = fr.to(dev)
    d = wt.make_desc(fr.width, fr.height, J, wt.F32, flags, tile[0], tile[1])
    f = wt.make_frags(g.pixel, g.z, g.alpha, g.tile_offsets, g.r, g.g, g.b)
    out = torch.empty(fr.P, 4, device=dev)
    acc = torch.full((fr.P, 5), float("nan"), device=dev)
    wt.wt_build_resolve(d, f, out, bg=(0.2, 0.4, 0.6), accum=acc)
    gout = torch.randn(fr.P, 4, device=dev, generator=torch.Generator(dev).manual_seed(J))
    res = []
    for a in (None, acc):
        ga = torch.full((fr.n,), float("nan"), device=dev)
        gc = torch.full((3, fr.n), float("nan"), device=dev)
        wt.wt_backward(d, f, gout, ga, gc, bg=(0.2, 0.4, 0.6), accum=a)
        res.append((ga, gc))
    assert wt.wt_get_error() == 0
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
    # the stored sums are the resolve's: S exact, ratios R/W as wt_resolve's
    h = acc.double().cpu().numpy()
    np.testing.assert_allclose(h[:, 4], _ref_S(fr), rtol=1e-5, atol=1e-6)


def _ref_S(fr):
    h = fr.numpy()
    a = -np.log1p(-np.clip(h["alpha"].astype(np.float64), 0, 1 - 2 ** -20))
    return np.bincount(h["pixel"].astype(np.int64), weights=a, minlength=fr.P)


def test_autograd_function_matches_direct_call():
    fr = synth.uniform_frame(48, 32, 10.0, 40, alpha_range=(0.05, 0.5), J=4, seed=8)
    dev = torch.device("cuda")
    g = fr.to(dev)
    d = wt.make_desc(fr.width, fr.height, 4)
    alpha = g.alpha.clone().requires_grad_(True)
    r, gg, b = (t.clone().requires_grad_(True) for t in (g.r, g.g, g.b))
    out = wt.WaveletOIT.apply(g.pixel, g.z, alpha, r, gg, b, g.tile_offsets, d, (0.5, 0.5, 0.5))
    target = torch.rand(fr.P, 4, device=dev, generator=torch.Generator(dev).manual_seed(3))
    loss = ((out - target) ** 2).sum()
    loss.backward()
    gout = (2 * (out - target)).detach().cpu().numpy()
    ra, rc = _ref_grad(fr, gout)
    _close(alpha.grad.double().cpu().numpy(), ra)
    _close(torch.stack([r.grad, gg.grad, b.grad], 1).double().cpu().numpy(), rc)


def test_diff512_batch_finite_differences():
    """16 frames of 512x512 (stacked as one 512x8192 image: pixels and tiles
    are independent), L2 loss against a seeded target; dL/dalpha and dL/drgb
    on 512 seeded sampled fragments against FP64 central differences of the
    oracle composite of each fragment's pixel."""
    dev = torch.device("cuda")
    fr = synth.diff512(seed=0, device=dev, width=512, height=512 * 16)
    d = wt.make_desc(fr.width, fr.height, 4)
    f = wt.make_frags(fr.pixel, fr.z, fr.alpha, fr.tile_offsets, fr.r, fr.g, fr.b)
    out = torch.empty(fr.P, 4, device=dev)
    acc = torch.empty(fr.P, 5, device=dev)
    wt.wt_build_resolve(d, f, out, None, None, accum=acc)
    target = torch.rand(fr.P, 4, device=dev, generator=torch.Generator(dev).manual_seed(5))
    target[:, 3] = out[:, 3]  # RGB loss only
    gout = (2 * (out - target)).contiguous()
    ga = torch.empty(fr.n, device=dev)
    gc = torch.empty(3, fr.n, device=dev)
    wt.wt_backward(d, f, gout, ga, gc)
    # the autograd path (the forward's pixel sums) gives the same gradients
    ga2, gc2 = torch.empty_like(ga), torch.empty_like(gc)
    wt.wt_backward(d, f, gout, ga2, gc2, accum=acc)
    assert wt.wt_get_error() == 0
    assert torch.equal(ga, ga2) and torch.equal(gc, gc2)
    del ga2, gc2
    rng = np.random.default_rng(512)
    sample = np.sort(rng.choice(fr.n, 512, replace=False))
    st = torch.from_numpy(sample).to(dev)
    ga_s = ga[st].double().cpu().numpy()
    gc_s = gc[:, st].double().cpu().numpy().T
    fd_a = np.zeros(512)
    fd_c = np.zeros((512, 3))
    pix = fr.pixel[st].long()
    for k in range(512):
        # the fragment's own pixel is an exact sub-problem (pixels are independent)
        idx, _ = synth.pixel_subset(fr, pix[k:k + 1])
        h = {kk: getattr(fr, kk)[idx].cpu().numpy() for kk in ("z", "alpha", "r", "g", "b")}
        j = int((idx == int(sample[k])).nonzero()[0, 0])
        loc = np.zeros(len(idx), np.uint32)
        tgt = target[pix[k]].double().cpu().numpy()

        def loss_of(al, cols):
            o = oracle.composite(loc, h["z"], al, cols, 1, 4)
            return ((o[0, :3] - tgt[:3]) ** 2).sum()

        cols = [h["r"], h["g"], h["b"]]
        hstep = np.float32(2.0 ** -12)
        ap, am = h["alpha"].copy(), h["alpha"].copy()
        ap[j] += hstep
        am[j] -= hstep
        fd_a[k] = (loss_of(ap, cols) - loss_of(am, cols)) / (float(ap[j]) - float(am[j]))
        for ch in range(3):
            cp = [c.copy() for c in cols]
            cm = [c.copy() for c in cols]
            cp[ch][j] += hstep
            cm[ch][j] -= hstep
            fd_c[k, ch] = (loss_of(h["alpha"], cp) - loss_of(h["alpha"], cm)) / \
                (float(cp[ch][j]) - float(cm[ch][j]))
    # central differences on float32 inputs: second-order truncation + the
    # rounding of the perturbed input bound the reference to ~1e-5 relative
    _close(ga_s, fd_a, rel=2e-3, absfrac=2e-4)
    _close(gc_s, fd_c, rel=1e-3, absfrac=1e-5)
