"""Serving with continuous batching on the GPU: results equal the single-frame
path, a frame's result is the same alone and in a mix of concurrent frames,
admission respects the byte cap (bounded waits time out while memory is held),
and bad requests are refused on the host."""
import time

import numpy as np
import pytest
import torch

import oracle
import paper_2201_00094_gb300 as wt
import synth

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


def _frame(w, h, lam, seed):
    return synth.serve_frame(w, h, lam, seed, device=DEV)


def _submit(srv, fr, dtype=wt.BF16):
    d = wt.make_desc(fr.width, fr.height, 4, dtype)
    f = wt.make_frags(fr.pixel, fr.z, fr.alpha, fr.tile_offsets, fr.r, fr.g, fr.b)
    out = torch.full((fr.P, 4), float("nan"), device=DEV)
    rid = srv.submit(d, f, out, keep=fr)
    return rid, out


def _direct(fr, dtype=wt.BF16):
    d = wt.make_desc(fr.width, fr.height, 4, dtype)
    f = wt.make_frags(fr.pixel, fr.z, fr.alpha, fr.tile_offsets, fr.r, fr.g, fr.b)
    out = torch.empty(fr.P, 4, device=DEV)
    wt.wt_build_resolve(d, f, out, None, None)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("dtype", [wt.F32, wt.BF16, wt.SE16])
def test_served_frame_equals_direct_call_and_oracle(dtype):
    """A served frame is the direct call's result bit for bit (every tile is
    computed from order-independent integer bins in one CTA, whatever else
    shares the launch), and matches the FP64 oracle: at 1e-4 with FP32
    storage; with SE16 at 1e-4 against the oracle's own encoding and within
    2e-3 of the unquantised composite; with BF16 within BF16's derived bound
    u (1 + J/2) S_p + 1e-4 (u = 2^-8) on every pixel -- this frame's
    opacities reach 0.6, and BF16 misses 2e-3 on some pixels of fewer than 32
    fragments here -- with the share within 2e-3 asserted above 99%."""
    fr = _frame(333, 197, 12.0, seed=1)
    with wt.Server(J=4, coeff_dtype=dtype, max_slots=4, mem_cap_bytes=1 << 30,
                   step_tiles=64) as srv:
        rid, out = _submit(srv, fr, dtype)
        assert srv.wait(rid, 20_000_000)
        info = srv.query(rid)
        assert info.state == 2 and info.done_us >= info.admit_us >= info.submit_us >= 0
        assert info.coeff
        srv.release(rid)
    assert torch.equal(out, _direct(fr, dtype))
    h = fr.to("cpu").numpy()
    rgb = (h["r"], h["g"], h["b"])
    exact = oracle.composite(h["pixel"], h["z"], h["alpha"], rgb, fr.P, 4)
    got = out.cpu().numpy().astype(np.float64)
    err = np.abs(got - exact).max(axis=1)
    if dtype == wt.F32:
        assert err.max() <= 1e-4
    elif dtype == wt.SE16:
        c32 = oracle.build_coeffs(h["pixel"], h["z"], h["alpha"], fr.P, 4).astype(np.float32)
        enc = oracle.se16_decode(*oracle.se16_encode(c32, 4), 4)
        ref = oracle.resolve(h["pixel"], h["z"], h["alpha"], rgb, fr.P, 4, enc)[0]
        assert np.abs(got - ref).max() <= 1e-4
        assert err.max() <= 2e-3
    else:
        ac = np.minimum(h["alpha"].astype(np.float64), 1 - 2.0 ** -20)
        S = np.bincount(h["pixel"].astype(np.int64), weights=-np.log1p(-ac), minlength=fr.P)
        assert (err <= 2.0 ** -8 * 3 * S + 1e-4).all()
        assert np.mean(err <= 2e-3) >= 0.99
    assert wt.wt_get_error() == 0


@pytest.mark.parametrize("dtype", [wt.BF16, wt.F32, wt.SE16])
def test_same_result_alone_and_in_mix(dtype):
    """A frame served alone and the same frame served among 24 concurrent
    frames of other sizes and depths give the same composite: bit for bit, as
    the build's fixed-point bins make every tile independent of fragment order
    and of what else shares the launch."""
    probe = _frame(640, 360, 20.0, seed=7)
    with wt.Server(J=4, coeff_dtype=dtype, max_slots=8, mem_cap_bytes=8 << 30,
                   step_tiles=2048) as srv:
        rid, out_alone = _submit(srv, probe, dtype)
        assert srv.wait(rid, 20_000_000)
        srv.release(rid)
        others = [_frame(*synth.SERVE_SIZES[k % 3], 2.0 + 4.0 * (k % 8), seed=100 + k)
                  for k in range(24)]
        ids = []
        for k, fr in enumerate(others):
            ids.append(_submit(srv, fr, dtype))
            if k == 11:
                pid, out_mix = _submit(srv, probe, dtype)   # arrives while others run
        for rid2, _ in ids:
            assert srv.wait(rid2, 60_000_000)
            srv.release(rid2)
        assert srv.wait(pid, 60_000_000)
        srv.release(pid)
        for (rid2, o), fr in zip(ids, others):
            assert torch.equal(o, _direct(fr, dtype))
    assert torch.equal(out_alone, out_mix)
    assert torch.isfinite(out_mix).all()


def test_admission_waits_for_memory_and_times_out():
    a = _frame(512, 512, 8.0, seed=3)
    b = _frame(512, 512, 8.0, seed=4)
    cap = a.n * 24 + 512 * 512 * (16 * 2 + 16) + 200_000  # room for one frame only
    with wt.Server(J=4, coeff_dtype=wt.BF16, max_slots=4, mem_cap_bytes=cap,
                   step_tiles=256) as srv:
        ra, oa = _submit(srv, a)
        rb, ob = _submit(srv, b)
        assert srv.wait(ra, 20_000_000)
        # b cannot be admitted while a is held: a bounded wait runs out
        assert not srv.wait(rb, 200_000)
        assert srv.query(rb).state == 0
        assert srv.stats()["queued"] == 1
        srv.release(ra)
        assert srv.wait(rb, 20_000_000)
        srv.release(rb)
        assert srv.stats()["used_bytes"] == 0
    assert torch.equal(ob, _direct(b))


def test_refused_requests():
    fr = _frame(64, 64, 4.0, seed=5)
    with wt.Server(J=4, coeff_dtype=wt.BF16, max_slots=2, mem_cap_bytes=1 << 20,
                   step_tiles=64) as srv:
        f = wt.make_frags(fr.pixel, fr.z, fr.alpha, fr.tile_offsets, fr.r, fr.g, fr.b)
        out = torch.empty(fr.P, 4, device=DEV)
        with pytest.raises(wt.WtError) as e:   # J differs from the server's
            srv.submit(wt.make_desc(64, 64, 5, wt.BF16), f, out)
        assert e.value.status == 2
        with pytest.raises(wt.WtError) as e:   # storage type differs
            srv.submit(wt.make_desc(64, 64, 4, wt.F32), f, out)
        assert e.value.status == 2
        big = _frame(1024, 1024, 4.0, seed=6)
        fb = wt.make_frags(big.pixel, big.z, big.alpha, big.tile_offsets, big.r, big.g, big.b)
        with pytest.raises(wt.WtError) as e:   # larger than the whole cap
            srv.submit(wt.make_desc(1024, 1024, 4, wt.BF16), fb,
                       torch.empty(big.P, 4, device=DEV))
        assert e.value.status == 6
        with pytest.raises(wt.WtError):        # release of an unknown request
            srv.release(12345)


def test_many_small_requests_complete_in_order_of_work():
    with wt.Server(J=4, coeff_dtype=wt.F16, max_slots=16, mem_cap_bytes=2 << 30,
                   step_tiles=512) as srv:
        frames = [_frame(96 + 16 * k, 64 + 8 * k, 4.0 + k, seed=200 + k) for k in range(20)]
        subs = []
        for fr in frames:
            d = wt.make_desc(fr.width, fr.height, 4, wt.F16)
            f = wt.make_frags(fr.pixel, fr.z, fr.alpha, fr.tile_offsets, fr.r, fr.g, fr.b)
            out = torch.empty(fr.P, 4, device=DEV)
            subs.append((srv.submit(d, f, out, keep=fr), out, fr))
        for rid, out, fr in subs:
            assert srv.wait(rid, 30_000_000)
            srv.release(rid)
            assert torch.equal(out, _direct(fr, wt.F16))
