"""The C-ABI library loads, exports every entry point include/wt.h declares,
and rejects bad arguments on the host (no GPU needed: argument checks run
before any CUDA call)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2201_00094_gb300 as wt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(wt.library_path()):
        from paper_2201_00094_gb300 import build_lib
        build_lib.build()
    return wt.lib()


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(wt_[a-z_0-9]+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(L):
    declared = _declared()
    assert {"wt_build", "wt_resolve", "wt_composite"} <= declared
    out = subprocess.run(["nm", "-D", "--defined-only", wt.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (wt_[a-z_0-9]+)$", out, flags=re.M))
    missing = declared - exported
    assert not missing, missing
    for name in declared:
        getattr(L, name)


def test_binding_passes_as_many_arguments_as_the_header_declares(L):
    """Every entry point the binding calls takes, in include/wt.h, exactly the
    number of arguments the binding passes (a call with one too few or too
    many would hand the library a shifted pointer)."""
    txt = ""
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt += open(os.path.join(ROOT, "include", h)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    checked = 0
    for name, params in re.findall(r"\b(wt_[a-z_0-9]+)\s*\(([^)]*)\)\s*;", txt):
        params = params.strip()
        count = 0 if params in ("", "void") else params.count(",") + 1
        argtypes = getattr(getattr(L, name), "argtypes", None)
        if argtypes is None:  # not called through the binding
            continue
        assert len(argtypes) == count, (name, count, len(argtypes))
        checked += 1
    assert checked >= 30


def test_struct_layout_matches_header():
    assert ctypes.sizeof(wt.WtDesc) == 32
    assert ctypes.sizeof(wt.WtFrags) == 64


def test_host_queries(L):
    d = wt.make_desc(1920, 1080, 4)
    assert wt.wt_coeff_bytes(d) == 1920 * 1080 * 16 * 4
    assert wt.wt_num_tiles(d) == 120 * 68
    d = wt.make_desc(3840, 2160, 5, wt.BF16)
    assert wt.wt_coeff_bytes(d) == 3840 * 2160 * 32 * 2
    d = wt.make_desc(53, 37, 3, tile_w=7, tile_h=3)
    assert wt.wt_num_tiles(d) == 8 * 13
    assert wt.wt_version().startswith("wt-gb300")


@pytest.mark.parametrize("bad", [
    dict(width=0), dict(height=-1), dict(J=0), dict(tile_w=0), dict(tile_w=32, tile_h=16),
    dict(coeff_dtype=7), dict(flags=1 << 9), dict(width=65536, height=65536)])
def test_bad_descriptor_rejected_on_host(L, bad):
    kw = dict(width=64, height=64, J=4, coeff_dtype=wt.F32, flags=wt.DEFAULT_FLAGS, tile_w=16,
              tile_h=16)
    kw.update(bad)
    d = wt.make_desc(**kw)
    assert L.wt_coeff_bytes(ctypes.byref(d)) == 0
    fr = wt.WtFrags()
    st = L.wt_build(ctypes.byref(d), ctypes.byref(fr), ctypes.c_void_p(16), None, None, None)
    assert st == 1


def test_unsupported_J_and_flags(L):
    d = wt.make_desc(64, 64, 7)
    fr = wt.WtFrags()
    assert L.wt_build(ctypes.byref(d), ctypes.byref(fr), ctypes.c_void_p(16), None, None, None) == 2
    # J = 6 is accepted (64 coefficients per pixel); these frags are then refused as arguments
    d6 = wt.make_desc(64, 64, 6)
    assert L.wt_coeff_bytes(ctypes.byref(d6)) == 64 * 64 * 64 * 4
    assert L.wt_build(ctypes.byref(d6), ctypes.byref(fr), ctypes.c_void_p(16), None, None, None) == 1
    d = wt.make_desc(64, 64, 4, flags=wt.DEFAULT_FLAGS | wt.ACCUMULATE)
    bg = (ctypes.c_float * 3)(0.5, 0.5, 0.5)
    st = L.wt_build_resolve(ctypes.byref(d), ctypes.byref(fr), None, None, None, bg,
                            ctypes.c_void_p(16), None, None)
    assert st == 2


def test_bad_fragment_pointers_rejected_on_host(L):
    d = wt.make_desc(64, 64, 4)
    fr = wt.WtFrags(n=10, pixel=None, z=16, alpha=16, tile_offsets=16)
    assert L.wt_build(ctypes.byref(d), ctypes.byref(fr), ctypes.c_void_p(16), None, None, None) == 1
    fr = wt.WtFrags(n=10, pixel=20, z=16, alpha=16, tile_offsets=16)  # misaligned
    assert L.wt_build(ctypes.byref(d), ctypes.byref(fr), ctypes.c_void_p(16), None, None, None) == 1
    fr = wt.WtFrags(n=10, pixel=16, z=16, alpha=16, tile_offsets=16)  # resolve needs rgb
    assert L.wt_resolve(ctypes.byref(d), ctypes.byref(fr), ctypes.c_void_p(16), None, None,
                        ctypes.c_void_p(16), None) == 1
    assert L.wt_get_error(None, None) == 1


def test_resolve_totals_rejected_on_host(L):
    """The build's per-pixel totals: a misaligned array is refused, and so is
    using them in an accumulating resolve (they cover every batch of a frame)."""
    fr = wt.WtFrags(n=10, pixel=16, z=16, alpha=16, r=16, g=16, b=16, tile_offsets=16)
    v, bad = ctypes.c_void_p(16), ctypes.c_void_p(18)
    bg = (ctypes.c_float * 3)(0.5, 0.5, 0.5)
    d = wt.make_desc(64, 64, 4)
    assert L.wt_build(ctypes.byref(d), ctypes.byref(fr), v, None, bad, None) == 1
    assert L.wt_resolve(ctypes.byref(d), ctypes.byref(fr), v, None, bad, v, None) == 1
    assert L.wt_resolve_composite(ctypes.byref(d), ctypes.byref(fr), v, None, bad, None, bg, v, None) == 1
    da = wt.make_desc(64, 64, 4, flags=wt.DEFAULT_FLAGS | wt.ACCUMULATE)
    assert L.wt_resolve(ctypes.byref(da), ctypes.byref(fr), v, None, v, v, None) == 2
    assert L.wt_resolve_composite(ctypes.byref(da), ctypes.byref(fr), v, None, v, None, bg, v, None) == 2


def test_coloured_fragment_pointers_rejected_on_host(L):
    """The coloured call reads every fragment array and the three opacity
    arrays as 16-byte vectors: a misaligned one is refused before any launch."""
    d = wt.make_desc(64, 64, 4)
    bg = (ctypes.c_float * 3)(0.5, 0.5, 0.5)
    v = ctypes.c_void_p(16)
    for bad in range(8):
        ptrs = [16] * 8
        ptrs[bad] = 20
        fr = wt.WtFrags(n=10, pixel=ptrs[0], z=ptrs[1], alpha=16, r=ptrs[2], g=ptrs[3], b=ptrs[4],
                        tile_offsets=16)
        a = [ctypes.c_void_p(x) for x in ptrs[5:]]
        st = L.wt_build_resolve_rgb(ctypes.byref(d), ctypes.byref(fr), *a, v, 0, None, bg, v, None)
        assert st == 1, bad
    fr = wt.WtFrags(n=10, pixel=16, z=16, alpha=16, r=16, g=16, b=16, tile_offsets=16)
    assert L.wt_build_resolve_rgb(ctypes.byref(d), ctypes.byref(fr), v, v, v, v, 0, None, bg, None, None) == 1


def test_backward_refuses_grad_alpha_overlapping_an_input(L):
    """grad_alpha holds intermediate values while the fragments are still being
    read: an overlap with any input array or with grad_rgb is refused before any
    launch."""
    d = wt.make_desc(64, 64, 4)
    bg = (ctypes.c_float * 3)(0.5, 0.5, 0.5)
    fr = wt.WtFrags(n=10, pixel=0x10000, z=0x20000, alpha=0x30000, r=0x40000, g=0x50000, b=0x60000,
                    tile_offsets=0x70000)
    gout, grgb = ctypes.c_void_p(0x80000), ctypes.c_void_p(0x90000)
    for ga in (0x30000, 0x30000 + 36, 0x10000 - 8, 0x60000, 0x70000 + 8, 0x80000 + 64, 0x90000 + 100):
        st = L.wt_backward(ctypes.byref(d), ctypes.byref(fr), None, bg, gout, None, ctypes.c_void_p(ga), grgb,
                           None)
        assert st == 1, hex(ga)
    acc = ctypes.c_void_p(0xA0000)  # the forward's pixel sums, 64 * 64 * 20 bytes
    for ga in (0xA0000, 0xA0000 + 64 * 64 * 20 - 4):
        st = L.wt_backward(ctypes.byref(d), ctypes.byref(fr), None, bg, gout, acc, ctypes.c_void_p(ga), grgb,
                           None)
        assert st == 1, hex(ga)
    st = L.wt_backward(ctypes.byref(d), ctypes.byref(fr), None, bg, gout, ctypes.c_void_p(0xA0002),
                       ctypes.c_void_p(0xC0000), grgb, None)  # misaligned sums
    assert st == 1


def test_status_strings(L):
    for s in range(8):
        assert L.wt_status_string(s)


def test_binding_requires_cuda_tensors():
    import torch
    with pytest.raises(ValueError):
        wt.make_frags(torch.zeros(4, dtype=torch.int32), torch.zeros(4), torch.zeros(4),
                      torch.zeros(2, dtype=torch.int64))


def test_coefficient_bytes_of_every_storage_type(L):
    """P * 2^J values of 4 or 2 bytes; the shared-exponent type adds one byte per pixel."""
    for J in (1, 4, 6):
        for dt, per in ((wt.F32, 4), (wt.BF16, 2), (wt.F16, 2), (wt.SE16, 2)):
            d = wt.make_desc(33, 7, J, dt)
            want = 33 * 7 * (1 << J) * per + (33 * 7 if dt == wt.SE16 else 0)
            assert L.wt_coeff_bytes(ctypes.byref(d)) == want == wt.coeff_storage_bytes(d)
    assert L.wt_coeff_bytes(ctypes.byref(wt.make_desc(33, 7, 4, 4))) == 0  # unknown type
