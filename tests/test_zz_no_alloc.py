"""wt_build_resolve_batch_static: the allocation-free batch entry point.

Callers that cannot allocate device memory when they submit work (a renderer
that reserves its whole device budget at start-up, or a real-time loop where
a cudaMalloc / cudaFree could synchronise the device and stall other work) use
this call; its scratch is a fixed array inside the library.  Checked through
the C ABI against wt_build_resolve, frame by frame, on two calls in a row (the
second reuses the scratch the first left behind).  Collected last on purpose,
and independent of every other test, so it passes alone in a fresh process."""
import pytest
import torch

import paper_2201_00094_gb300 as wt
import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


def _batch(sizes, seed, J=4, dtype=wt.F32, flags=wt.DEFAULT_FLAGS, tile=(16, 16)):
    frames = [synth.uniform_frame(w, h, lam, 64, alpha_range=(0.05, 0.6), J=J, seed=seed + i,
                                  device=DEV, tile_w=tile[0], tile_h=tile[1])
              for i, (w, h, lam) in enumerate(sizes)]
    descs = [wt.make_desc(f.width, f.height, J, dtype, flags, tile[0], tile[1]) for f in frames]
    frags = [wt.make_frags(f.pixel, f.z, f.alpha, f.tile_offsets, f.r, f.g, f.b) for f in frames]
    return frames, descs, frags


def _reference(fr, d, f, bg):
    out = torch.empty(fr.P, 4, device=DEV)
    wt.wt_build_resolve(d, f, out, None, None, bg=bg)
    return out


# the tolerances of the other tests: FP32 storage 1e-5 between two runs of the
# same arithmetic, 16-bit storage its 2e-3 target
TOL = {wt.F32: 1e-5, wt.BF16: 2e-3, wt.F16: 2e-3}


@pytest.mark.parametrize("dtype", [wt.F32, wt.BF16, wt.F16])
@pytest.mark.parametrize("J", [4, 5])
def test_static_batch_matches_build_resolve_twice(dtype, J):
    bgs = [(0.5, 0.5, 0.5), (0.1, 0.2, 0.3), (0.9, 0.8, 0.7), (0.0, 1.0, 0.5), (0.3, 0.3, 0.3)]
    for call, sizes in enumerate([[(333, 197, 9.0), (64, 64, 4.0), (257, 31, 20.0)],
                                  [(120, 90, 12.0), (500, 301, 6.0), (17, 33, 3.0),
                                   (1024, 16, 30.0), (200, 200, 1.0)]]):
        frames, descs, frags = _batch(sizes, seed=10 * call + J, J=J, dtype=dtype)
        outs = [torch.full((f.P, 4), float("nan"), device=DEV) for f in frames]
        wt.wt_build_resolve_batch_static(descs, frags, outs, bgs[:len(frames)])
        torch.cuda.synchronize()
        for k, (fr, d, f) in enumerate(zip(frames, descs, frags)):
            ref = _reference(fr, d, f, bgs[k])
            assert torch.isfinite(outs[k]).all()
            assert (outs[k] - ref).abs().max().item() <= TOL[dtype]
    assert wt.wt_get_error() == 0


@pytest.mark.parametrize("flags", [wt.SELF_EXCLUDE | wt.INTERP_LINEAR, wt.RESOLVE_NORMALIZED, 0])
def test_static_batch_other_readings_and_tile(flags):
    """Readings other than the default and 192 x 1 row tiles (the bench's)."""
    for call in range(2):
        frames, descs, frags = _batch([(400, 60, 10.0), (191, 7, 3.0)], seed=200 + flags + call,
                                      J=5, flags=flags, tile=(192, 1))
        outs = [torch.full((f.P, 4), float("nan"), device=DEV) for f in frames]
        wt.wt_build_resolve_batch_static(descs, frags, outs)
        torch.cuda.synchronize()
        for fr, d, f, o in zip(frames, descs, frags, outs):
            assert (o - _reference(fr, d, f, (0.5, 0.5, 0.5))).abs().max().item() <= 1e-5
    assert wt.wt_get_error() == 0


def test_static_batch_rejects_oversized_and_mixed_batches():
    frames, descs, frags = _batch([(32, 32, 2.0)], seed=99)
    out = torch.empty(frames[0].P, 4, device=DEV)
    with pytest.raises(wt.WtError) as e:  # more frames than the scratch holds
        wt.wt_build_resolve_batch_static(descs * 65, frags * 65, [out] * 65)
    assert e.value.status == 1
    d5 = wt.make_desc(32, 32, 5, wt.F32)
    with pytest.raises(wt.WtError) as e:  # frames must share J
        wt.wt_build_resolve_batch_static([descs[0], d5], frags * 2, [out, out])
    assert e.value.status == 2
