"""Host logic of the Python binding that needs no GPU: the size checks it
applies before every call (the C ABI takes bare pointers)."""
import pytest
import torch

import paper_2201_00094_gb300 as wt


def test_need_counts_elements():
    wt._need(None, "x", 10)  # optional buffers
    wt._need(torch.empty(10), "x", 10)
    wt._need(torch.empty(2, 5), "x", 10)
    with pytest.raises(ValueError, match="x holds 9 elements"):
        wt._need(torch.empty(9), "x", 10)


def test_pixel_buffers_follow_the_descriptor():
    d = wt.make_desc(7, 5, 3)  # P = 35, C = 8
    P = 35
    wt._check_pixel_buffers(d, coeff=torch.empty(P, 8), zmin=torch.empty(P), accum=torch.empty(P, 5),
                            out=torch.empty(P, 4), bg_img=torch.empty(P, 3))
    for kw in ({"coeff": torch.empty(P, 7)}, {"zmin": torch.empty(P - 1)}, {"accum": torch.empty(P, 4)},
               {"out": torch.empty(P - 1, 4)}, {"bg_img": torch.empty(P, 2)}):
        with pytest.raises(ValueError):
            wt._check_pixel_buffers(d, **kw)
    # the coloured call's FP32 planes hold three coefficient rows per pixel
    wt._check_pixel_buffers(d, coeff=torch.empty(3, P, 8), coeff_per_pixel=24)
    with pytest.raises(ValueError):
        wt._check_pixel_buffers(d, coeff=torch.empty(P, 8), coeff_per_pixel=24)


def test_tile_offsets_must_cover_the_descriptor_tiles():
    d = wt.make_desc(40, 20, 4, tile_w=16, tile_h=16)  # 3 x 2 tiles
    f = wt.WtFrags(0, None, None, None, None, None, None, None)
    wt._check_frags(d, f)  # built without make_frags: nothing recorded, nothing checked
    f._tile_offsets = 7
    wt._check_frags(d, f)
    f._tile_offsets = 6
    with pytest.raises(ValueError, match="6 tiles"):
        wt._check_frags(d, f)


def test_shared_exponent_buffers_are_checked_in_bytes():
    """SE16 coefficient buffers are bytes: P * C two-byte mantissas, then P
    exponent bytes; a buffer of another storage type is refused."""
    d = wt.make_desc(7, 5, 3, wt.SE16)  # P = 35, C = 8
    assert wt.coeff_storage_bytes(d) == 35 * 8 * 2 + 35
    wt._check_pixel_buffers(d, coeff=torch.empty(35 * 17, dtype=torch.uint8))
    with pytest.raises(ValueError, match="bytes"):
        wt._check_pixel_buffers(d, coeff=torch.empty(35 * 17 - 1, dtype=torch.uint8))
    with pytest.raises(ValueError, match="dtype"):
        wt._check_pixel_buffers(d, coeff=torch.empty(35, 8, dtype=torch.bfloat16))
    with pytest.raises(ValueError, match="dtype"):
        wt._check_pixel_buffers(wt.make_desc(7, 5, 3, wt.BF16), coeff=torch.empty(35, 8))


def test_static_batch_checks_every_frame_before_the_call():
    """wt_build_resolve_batch_static takes bare pointers for up to 64 frames:
    the binding refuses lists of different lengths and an undersized output
    or tile table of any frame before anything reaches the library."""
    d = wt.make_desc(8, 4, 4, tile_w=8, tile_h=1)  # P = 32, 4 tiles
    f = wt.WtFrags(0, None, None, None, None, None, None, None)
    f._tile_offsets = 5
    ok = torch.empty(32, 4)
    with pytest.raises(ValueError, match="one entry per frame"):
        wt.wt_build_resolve_batch_static([d, d], [f], [ok, ok])
    with pytest.raises(ValueError, match="one entry per frame"):
        wt.wt_build_resolve_batch_static([d], [f], [ok], bgs=[(0.5, 0.5, 0.5)] * 2)
    with pytest.raises(ValueError, match="out holds"):
        wt.wt_build_resolve_batch_static([d, d], [f, f], [ok, torch.empty(31, 4)])
    short = wt.WtFrags(0, None, None, None, None, None, None, None)
    short._tile_offsets = 4
    with pytest.raises(ValueError, match="4 tiles"):
        wt.wt_build_resolve_batch_static([d, d], [f, short], [ok, ok])


def test_totals_and_pixel_sums_are_checked_before_the_call():
    """The optional per-pixel totals of wt_build / wt_resolve and the pixel sums
    of wt_build_resolve / wt_backward are bare pointers too: undersized ones are
    refused before anything reaches the library."""
    d = wt.make_desc(7, 5, 3)  # P = 35, C = 8
    P = 35
    f = wt.WtFrags(0, None, None, None, None, None, None, None)
    coeff, out = torch.empty(P, 8), torch.empty(P, 4)
    with pytest.raises(ValueError, match="total"):
        wt.wt_build(d, f, coeff, total=torch.empty(P - 1))
    with pytest.raises(ValueError, match="total"):
        wt.wt_resolve(d, f, coeff, None, torch.empty(P, 5), total=torch.empty(P - 1))
    with pytest.raises(ValueError, match="total"):
        wt.wt_resolve_composite(d, f, coeff, None, out, total=torch.empty(P - 1))
    with pytest.raises(ValueError, match="accum"):
        wt.wt_build_resolve(d, f, out, accum=torch.empty(P, 4))
    with pytest.raises(ValueError, match="accum"):
        wt.wt_backward(d, f, torch.empty(P, 4), torch.empty(0), torch.empty(3, 0), accum=torch.empty(P - 1, 5))
