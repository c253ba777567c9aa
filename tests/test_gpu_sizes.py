"""The binding refuses tensors smaller than a call reads or writes (the C ABI
takes bare pointers, so the sizes are checked before the call)."""
import pytest
import torch

import paper_2201_00094_gb300 as wt
import synth
from wtcheck import desc_of, frags_of

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda")


def test_small_buffers_are_refused_before_the_call():
    fr = synth.uniform_frame(40, 20, 4.0, 20, J=4, seed=5, tile_w=16, tile_h=16)
    g = fr.to(DEV)
    d = desc_of(fr)
    f = frags_of(g)
    P = fr.P
    ok_out = torch.empty(P, 4, device=DEV)
    with pytest.raises(ValueError):
        wt.wt_build_resolve(d, f, torch.empty(P - 1, 4, device=DEV))
    with pytest.raises(ValueError):
        wt.wt_build_resolve(d, f, ok_out, torch.empty(P, 15, device=DEV))
    with pytest.raises(ValueError):
        wt.wt_build(d, f, torch.empty(P, 16, device=DEV), torch.empty(P - 1, device=DEV))
    with pytest.raises(ValueError):
        wt.wt_composite(d, torch.empty(P, 4, device=DEV), ok_out)
    with pytest.raises(ValueError):
        wt.wt_build_resolve_rgb(d, f, g.alpha, g.alpha, g.alpha[:-1], ok_out)
    with pytest.raises(ValueError):
        wt.wt_build_resolve_rgb(d, f, g.alpha, g.alpha, g.alpha, ok_out, torch.empty(P, 16, device=DEV))
    with pytest.raises(ValueError):
        wt.wt_composite_ca(d, torch.empty(P, 5, device=DEV), torch.empty(P, 3, device=DEV), ok_out,
                           torch.empty(P, 1, device=DEV))
    with pytest.raises(ValueError):  # tile offsets of another tiling
        wt.wt_build_resolve(wt.make_desc(fr.width, fr.height, 4, tile_w=8, tile_h=8), f, ok_out)
    with pytest.raises(ValueError):
        wt.make_frags(g.pixel[:-1], g.z, g.alpha, g.tile_offsets)
    # the right sizes go through
    wt.wt_build_resolve(d, f, ok_out, torch.empty(P, 16, device=DEV))
    assert wt.wt_get_error() == 0
