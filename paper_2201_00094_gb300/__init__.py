"""Python binding of libwt.so: GB300 Wavelet OIT (Aizenshtein, Smal & McGuire,
"Wavelet Transparency", 2021).

Argument marshalling only.  Every step of the method runs in the CUDA kernels
of libwt.so (built in-tree by ``build_lib.build()``); nothing here computes a
result and there is no CPU fallback.  If the library is missing, the first
call raises.

Tensors are torch CUDA tensors (device memory and streams only).  Calls are
asynchronous on ``stream`` (default: torch's current stream).  The names
follow the C ABI in include/wt.h.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

__all__ = [
    "F32", "BF16", "F16", "SE16", "coeff_buffer", "coeff_storage_bytes", "SELF_EXCLUDE", "INTERP_LINEAR", "RESOLVE_NORMALIZED", "ACCUMULATE",
    "DEFAULT_FLAGS", "WtDesc", "WtFrags", "WtError", "lib", "library_path", "make_desc",
    "make_frags", "coeff_torch_dtype", "wt_version", "wt_coeff_bytes", "wt_num_tiles", "wt_build",
    "wt_resolve", "wt_composite", "wt_resolve_composite", "wt_build_resolve", "wt_absorbance",
    "wt_get_error", "wt_backward", "WaveletOIT", "Server", "Planner", "WtServeConfig",
    "WtServeInfo", "wt_build_resolve_batch_static", "wt_bin_workspace_bytes", "wt_bin",
    "wt_depth_bounds", "wt_normalize_depth", "wt_build_resolve_tiles", "wt_build_resolve_single_pass",
    "WtParticles", "wt_raster", "RGB_F32", "RGB_E5B9G9R9", "wt_build_resolve_rgb", "wt_composite_ca", "WtTriangles", "wt_raster_tri",
]

F32, BF16, F16, SE16 = 0, 1, 2, 3
SELF_EXCLUDE, INTERP_LINEAR, RESOLVE_NORMALIZED, ACCUMULATE = 1, 2, 4, 8
DEFAULT_FLAGS = SELF_EXCLUDE | INTERP_LINEAR | RESOLVE_NORMALIZED

_DIR = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_DIR, "libwt.so")
_STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported", 3: "rejected input fragments",
           4: "timeout", 5: "CUDA error", 6: "over memory cap", 7: "busy"}
_TORCH_DTYPE = {F32: torch.float32, BF16: torch.bfloat16, F16: torch.float16, SE16: torch.uint8}


class WtError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn}: {_STATUS.get(status, status)} (status {status})")
        self.status = status


class WtDesc(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("J", ctypes.c_int32), ("coeff_dtype", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("reserved", ctypes.c_int32)]

    @property
    def P(self) -> int:
        return self.width * self.height

    @property
    def C(self) -> int:
        return 1 << self.J


class WtFrags(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("pixel", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("alpha", ctypes.c_void_p), ("r", ctypes.c_void_p), ("g", ctypes.c_void_p),
                ("b", ctypes.c_void_p), ("tile_offsets", ctypes.c_void_p)]


class WtParticles(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("cx", ctypes.c_void_p), ("cy", ctypes.c_void_p),
                ("radius", ctypes.c_void_p), ("z", ctypes.c_void_p), ("alpha", ctypes.c_void_p),
                ("r", ctypes.c_void_p), ("g", ctypes.c_void_p), ("b", ctypes.c_void_p)]


class WtTriangles(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("alpha", ctypes.c_void_p), ("r", ctypes.c_void_p), ("g", ctypes.c_void_p),
                ("b", ctypes.c_void_p)]


class WtServeConfig(ctypes.Structure):
    _fields_ = [("J", ctypes.c_int32), ("coeff_dtype", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32),
                ("max_slots", ctypes.c_int32), ("mem_cap_bytes", ctypes.c_int64),
                ("step_tiles", ctypes.c_int64)]


class WtServeInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("submit_us", ctypes.c_double), ("admit_us", ctypes.c_double),
                ("done_us", ctypes.c_double), ("coeff", ctypes.c_void_p)]


_lib: Optional[ctypes.CDLL] = None


def library_path() -> str:
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    """The loaded libwt.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is not built; run __graft_entry__.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(_LIB_PATH)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    D, Fr = ctypes.POINTER(WtDesc), ctypes.POINTER(WtFrags)
    sig = {
        "wt_version": ([], ctypes.c_char_p),
        "wt_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "wt_coeff_bytes": ([D], ctypes.c_size_t),
        "wt_num_tiles": ([D], i64),
        "wt_build": ([D, Fr, vp, vp, vp, vp], ctypes.c_int),
        "wt_resolve": ([D, Fr, vp, vp, vp, vp, vp], ctypes.c_int),
        "wt_composite": ([D, vp, vp, vp, vp, vp], ctypes.c_int),
        "wt_composite_ca": ([D, vp, vp, vp, ctypes.c_float, ctypes.c_int32, vp, vp], ctypes.c_int),
        "wt_resolve_composite": ([D, Fr, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "wt_build_resolve": ([D, Fr, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "wt_build_resolve_tiles": ([D, Fr, i64, i64, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "wt_build_resolve_single_pass": ([D, Fr, vp, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "wt_build_resolve_rgb": ([D, Fr, vp, vp, vp, vp, ctypes.c_int32, vp, vp, vp, vp], ctypes.c_int),
        "wt_absorbance": ([D, vp, i64, vp, vp, vp, vp, vp], ctypes.c_int),
        "wt_backward": ([D, Fr, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
        "wt_build_resolve_batch_static": ([D, Fr, vp, vp, ctypes.c_int32, vp], ctypes.c_int),
        "wt_get_error": ([vp, ctypes.POINTER(i64)], ctypes.c_int),
        "wt_raster_workspace_bytes": ([i64], ctypes.c_size_t),
        "wt_raster_count": ([D, ctypes.POINTER(WtParticles), vp, vp], ctypes.c_int),
        "wt_raster_emit": ([D, ctypes.POINTER(WtParticles), vp, i64, vp, vp, vp, vp, vp, vp, vp],
                           ctypes.c_int),
        "wt_raster_tri_count": ([D, ctypes.POINTER(WtTriangles), vp, vp], ctypes.c_int),
        "wt_raster_tri_emit": ([D, ctypes.POINTER(WtTriangles), vp, i64, vp, vp, vp, vp, vp, vp, vp],
                               ctypes.c_int),
        "wt_bin_workspace_bytes": ([D, i64], ctypes.c_size_t),
        "wt_bin": ([D, Fr, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp], ctypes.c_int),
        "wt_depth_bounds": ([D, Fr, vp, vp, vp], ctypes.c_int),
        "wt_normalize_depth": ([D, Fr, vp, vp, vp, vp], ctypes.c_int),
        "wt_serve_create": ([ctypes.POINTER(WtServeConfig), ctypes.POINTER(vp)], ctypes.c_int),
        "wt_serve_submit": ([vp, D, Fr, vp, vp, vp, ctypes.POINTER(i64)], ctypes.c_int),
        "wt_serve_wait": ([vp, i64, i64], ctypes.c_int),
        "wt_serve_query": ([vp, i64, ctypes.POINTER(WtServeInfo)], ctypes.c_int),
        "wt_serve_release": ([vp, i64], ctypes.c_int),
        "wt_serve_stats": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)],
                           ctypes.c_int),
        "wt_serve_destroy": ([vp], ctypes.c_int),
        "wt_planner_create": ([ctypes.c_int32, i64, i64], vp),
        "wt_planner_submit": ([vp, i64, i64], i64),
        "wt_planner_admit": ([vp, vp, ctypes.c_int32], ctypes.c_int32),
        "wt_planner_plan": ([vp, vp, vp, vp, ctypes.c_int32, vp, ctypes.POINTER(ctypes.c_int32)],
                            ctypes.c_int32),
        "wt_planner_release": ([vp, i64], ctypes.c_int32),
        "wt_planner_used": ([vp], i64),
        "wt_planner_destroy": ([vp], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


# ---------------------------------------------------------------- marshalling

def _stream(stream) -> Optional[int]:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev(t: Optional[torch.Tensor], name: str, dtypes) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.dtype not in dtypes:
        raise ValueError(f"{name} has dtype {t.dtype}, expected one of {dtypes}")
    return t.data_ptr()


def _call(name: str, *args) -> None:
    st = getattr(lib(), name)(*args)
    if st != 0:
        raise WtError(name, st)


def coeff_torch_dtype(coeff_dtype: int) -> torch.dtype:
    """Element type of a coefficient tensor: float32 / bfloat16 / float16
    [P, C], or uint8 bytes for SE16 (mantissas, then exponent bytes)."""
    return _TORCH_DTYPE[coeff_dtype]


def coeff_storage_bytes(desc: "WtDesc") -> int:
    """Bytes of a frame's coefficient buffer (the formula of wt_coeff_bytes)."""
    P, C = _pixels(desc), 1 << int(desc.J)
    dt = int(desc.coeff_dtype)
    return P * C * (4 if dt == F32 else 2) + (P if dt == SE16 else 0)


def coeff_buffer(desc: "WtDesc", device) -> torch.Tensor:
    """An uninitialised coefficient buffer for desc: [P, C] of the storage
    type, or [wt_coeff_bytes] uint8 for SE16."""
    dt = int(desc.coeff_dtype)
    if dt == SE16:
        return torch.empty(coeff_storage_bytes(desc), dtype=torch.uint8, device=device)
    return torch.empty(_pixels(desc), 1 << int(desc.J), dtype=_TORCH_DTYPE[dt], device=device)


def make_desc(width: int, height: int, J: int, coeff_dtype: int = F32,
              flags: int = DEFAULT_FLAGS, tile_w: int = 16, tile_h: int = 16) -> WtDesc:
    return WtDesc(width, height, tile_w, tile_h, J, coeff_dtype, flags, 0)


def make_frags(pixel: torch.Tensor, z: torch.Tensor, alpha: torch.Tensor,
               tile_offsets: torch.Tensor, r: Optional[torch.Tensor] = None,
               g: Optional[torch.Tensor] = None, b: Optional[torch.Tensor] = None) -> WtFrags:
    """Fragment stream descriptor.  The caller keeps the tensors alive."""
    f32 = (torch.float32,)
    n = int(z.numel())
    for t, name in ((pixel, "pixel"), (alpha, "alpha"), (r, "r"), (g, "g"), (b, "b")):
        _need(t, name, n)
    f = WtFrags(n, _dev(pixel, "pixel", (torch.int32, torch.uint32)),
                _dev(z, "z", f32), _dev(alpha, "alpha", f32), _dev(r, "r", f32),
                _dev(g, "g", f32), _dev(b, "b", f32),
                _dev(tile_offsets, "tile_offsets", (torch.int64,)))
    f._tile_offsets = int(tile_offsets.numel())  # checked against a descriptor's tile count
    return f


# Size checks: the C ABI takes bare pointers, so the binding checks that every
# tensor holds at least what the call reads or writes.
def _need(t: Optional[torch.Tensor], name: str, count: int) -> None:
    if t is not None and t.numel() < count:
        raise ValueError(f"{name} holds {t.numel()} elements; the call needs {count}")


def _pixels(desc: "WtDesc") -> int:
    return int(desc.width) * int(desc.height)


def _check_frags(desc: "WtDesc", frags: "WtFrags") -> None:
    have = getattr(frags, "_tile_offsets", None)
    if have is not None:
        ntiles = (-(-int(desc.width) // int(desc.tile_w))) * (-(-int(desc.height) // int(desc.tile_h)))
        if have < ntiles + 1:
            raise ValueError(f"tile_offsets holds {have} entries; the descriptor has {ntiles} tiles")


def _check_pixel_buffers(desc: "WtDesc", coeff=None, zmin=None, accum=None, out=None, bg_img=None,
                         coeff_per_pixel: Optional[int] = None) -> None:
    P = _pixels(desc)
    if coeff is not None and coeff_per_pixel is None:
        # mono storage: checked in bytes and against the descriptor's type
        want = _TORCH_DTYPE.get(int(desc.coeff_dtype))
        if want is not None and coeff.dtype != want:
            raise ValueError(f"coeff has dtype {coeff.dtype}; the descriptor's storage needs {want}")
        have = coeff.numel() * coeff.element_size()
        if have < coeff_storage_bytes(desc):
            raise ValueError(f"coeff holds {have} bytes; the call needs {coeff_storage_bytes(desc)}")
        coeff = None
    _need(coeff, "coeff", P * (coeff_per_pixel if coeff_per_pixel is not None else 1 << int(desc.J)))
    _need(zmin, "zmin", P)
    _need(accum, "accum", 5 * P)
    _need(out, "out", 4 * P)
    _need(bg_img, "bg_img", 3 * P)


def _bg(bg: Sequence[float]):
    return (ctypes.c_float * 3)(*[float(x) for x in bg])


_COEFF_DT = (torch.float32, torch.bfloat16, torch.float16, torch.uint8)


# ---------------------------------------------------------------- entry points

def wt_version() -> str:
    return lib().wt_version().decode()


def wt_coeff_bytes(desc: WtDesc) -> int:
    return int(lib().wt_coeff_bytes(ctypes.byref(desc)))


def wt_num_tiles(desc: WtDesc) -> int:
    return int(lib().wt_num_tiles(ctypes.byref(desc)))


def wt_build(desc: WtDesc, frags: WtFrags, coeff: torch.Tensor,
             zmin: Optional[torch.Tensor] = None, stream=None,
             total: Optional[torch.Tensor] = None) -> None:
    """total [P] float32, optional: each pixel's total step, for wt_resolve."""
    _check_frags(desc, frags)
    _check_pixel_buffers(desc, coeff=coeff, zmin=zmin)
    _need(total, "total", _pixels(desc))
    _call("wt_build", ctypes.byref(desc), ctypes.byref(frags), _dev(coeff, "coeff", _COEFF_DT),
          _dev(zmin, "zmin", (torch.float32,)), _dev(total, "total", (torch.float32,)), _stream(stream))


def wt_resolve(desc: WtDesc, frags: WtFrags, coeff: torch.Tensor, zmin: Optional[torch.Tensor],
               accum: torch.Tensor, stream=None, total: Optional[torch.Tensor] = None) -> None:
    _check_frags(desc, frags)
    _check_pixel_buffers(desc, coeff=coeff, zmin=zmin, accum=accum)
    _need(total, "total", _pixels(desc))
    _call("wt_resolve", ctypes.byref(desc), ctypes.byref(frags), _dev(coeff, "coeff", _COEFF_DT),
          _dev(zmin, "zmin", (torch.float32,)), _dev(total, "total", (torch.float32,)),
          _dev(accum, "accum", (torch.float32,)), _stream(stream))


def wt_composite(desc: WtDesc, accum: torch.Tensor, out: torch.Tensor,
                 bg: Sequence[float] = (0.5, 0.5, 0.5), bg_img: Optional[torch.Tensor] = None,
                 stream=None) -> None:
    _check_pixel_buffers(desc, accum=accum, out=out, bg_img=bg_img)
    _call("wt_composite", ctypes.byref(desc), _dev(accum, "accum", (torch.float32,)),
          _dev(bg_img, "bg_img", (torch.float32,)), _bg(bg), _dev(out, "out", (torch.float32,)),
          _stream(stream))


def wt_resolve_composite(desc: WtDesc, frags: WtFrags, coeff: torch.Tensor,
                         zmin: Optional[torch.Tensor], out: torch.Tensor,
                         bg: Sequence[float] = (0.5, 0.5, 0.5),
                         bg_img: Optional[torch.Tensor] = None, stream=None,
                         total: Optional[torch.Tensor] = None) -> None:
    _check_frags(desc, frags)
    _check_pixel_buffers(desc, coeff=coeff, zmin=zmin, out=out, bg_img=bg_img)
    _need(total, "total", _pixels(desc))
    _call("wt_resolve_composite", ctypes.byref(desc), ctypes.byref(frags),
          _dev(coeff, "coeff", _COEFF_DT), _dev(zmin, "zmin", (torch.float32,)),
          _dev(total, "total", (torch.float32,)), _dev(bg_img, "bg_img", (torch.float32,)), _bg(bg),
          _dev(out, "out", (torch.float32,)), _stream(stream))


def wt_build_resolve(desc: WtDesc, frags: WtFrags, out: torch.Tensor,
                     coeff: Optional[torch.Tensor] = None, zmin: Optional[torch.Tensor] = None,
                     bg: Sequence[float] = (0.5, 0.5, 0.5), bg_img: Optional[torch.Tensor] = None,
                     stream=None, accum: Optional[torch.Tensor] = None) -> None:
    """accum [P, 5] float32, optional: the pixel sums, for wt_backward."""
    _check_frags(desc, frags)
    _check_pixel_buffers(desc, coeff=coeff, zmin=zmin, out=out, bg_img=bg_img, accum=accum)
    _call("wt_build_resolve", ctypes.byref(desc), ctypes.byref(frags),
          _dev(coeff, "coeff", _COEFF_DT), _dev(zmin, "zmin", (torch.float32,)),
          _dev(bg_img, "bg_img", (torch.float32,)), _bg(bg), _dev(out, "out", (torch.float32,)),
          _dev(accum, "accum", (torch.float32,)), _stream(stream))


def wt_build_resolve_tiles(desc: WtDesc, frags: WtFrags, first_tile: int, num_tiles: int,
                           out: torch.Tensor, coeff: Optional[torch.Tensor] = None,
                           zmin: Optional[torch.Tensor] = None, bg: Sequence[float] = (0.5, 0.5, 0.5),
                           bg_img: Optional[torch.Tensor] = None, stream=None,
                           accum: Optional[torch.Tensor] = None) -> None:
    _check_frags(desc, frags)
    _check_pixel_buffers(desc, coeff=coeff, zmin=zmin, out=out, bg_img=bg_img, accum=accum)
    _call("wt_build_resolve_tiles", ctypes.byref(desc), ctypes.byref(frags), int(first_tile),
          int(num_tiles), _dev(coeff, "coeff", _COEFF_DT), _dev(zmin, "zmin", (torch.float32,)),
          _dev(bg_img, "bg_img", (torch.float32,)), _bg(bg), _dev(out, "out", (torch.float32,)),
          _dev(accum, "accum", (torch.float32,)), _stream(stream))


def wt_build_resolve_single_pass(desc: WtDesc, frags: WtFrags, coeff_prev: torch.Tensor,
                                 out: torch.Tensor, coeff: Optional[torch.Tensor] = None,
                                 zmin_prev: Optional[torch.Tensor] = None,
                                 zmin: Optional[torch.Tensor] = None, bg: Sequence[float] = (0.5, 0.5, 0.5),
                                 bg_img: Optional[torch.Tensor] = None, stream=None) -> None:
    """Resolves this frame against the previous frame's coefficients and
    builds this frame's coefficients in one pass (wt_build_resolve_single_pass)."""
    _check_frags(desc, frags)
    _check_pixel_buffers(desc, coeff=coeff_prev, zmin=zmin_prev, out=out, bg_img=bg_img)
    _check_pixel_buffers(desc, coeff=coeff, zmin=zmin)
    _call("wt_build_resolve_single_pass", ctypes.byref(desc), ctypes.byref(frags),
          _dev(coeff_prev, "coeff_prev", _COEFF_DT), _dev(zmin_prev, "zmin_prev", (torch.float32,)),
          _dev(coeff, "coeff", _COEFF_DT), _dev(zmin, "zmin", (torch.float32,)),
          _dev(bg_img, "bg_img", (torch.float32,)), _bg(bg), _dev(out, "out", (torch.float32,)),
          _stream(stream))


RGB_F32, RGB_E5B9G9R9 = 0, 1


def wt_build_resolve_rgb(desc: WtDesc, frags: WtFrags, alpha_r: torch.Tensor, alpha_g: torch.Tensor,
                         alpha_b: torch.Tensor, out: torch.Tensor, coeff: Optional[torch.Tensor] = None,
                         coeff_format: int = RGB_F32, bg: Sequence[float] = (0.5, 0.5, 0.5),
                         bg_img: Optional[torch.Tensor] = None, stream=None) -> None:
    """Coloured absorbance (wt_build_resolve_rgb): per-channel opacity, one
    depth; coeff is float32 [3, P, C] (RGB_F32, one plane per channel) or
    int32/uint32 [P, C] words (RGB_E5B9G9R9)."""
    f32 = (torch.float32,)
    cdt = f32 if coeff_format == RGB_F32 else (torch.int32, torch.uint32)
    _check_frags(desc, frags)
    for t, name in ((alpha_r, "alpha_r"), (alpha_g, "alpha_g"), (alpha_b, "alpha_b")):
        _need(t, name, int(frags.n))
    C = 1 << int(desc.J)
    _check_pixel_buffers(desc, coeff=coeff, out=out, bg_img=bg_img,
                         coeff_per_pixel=3 * C if coeff_format == RGB_F32 else C)
    _call("wt_build_resolve_rgb", ctypes.byref(desc), ctypes.byref(frags), _dev(alpha_r, "alpha_r", f32),
          _dev(alpha_g, "alpha_g", f32), _dev(alpha_b, "alpha_b", f32), _dev(coeff, "coeff", cdt),
          int(coeff_format), _dev(bg_img, "bg_img", f32), _bg(bg), _dev(out, "out", f32), _stream(stream))


def wt_composite_ca(desc: WtDesc, accum: torch.Tensor, bg_img: torch.Tensor, out: torch.Tensor,
                    offset: Optional[torch.Tensor] = None, dispersion: float = 0.5, taps: int = 5,
                    stream=None) -> None:
    """Composite with the chromatic-aberration background gather (wt_composite_ca):
    accum [P, 5] from wt_resolve, bg_img [P, 3], offset [P, 2] refraction offsets
    in pixels (None: no offset)."""
    f32 = (torch.float32,)
    _check_pixel_buffers(desc, accum=accum, out=out, bg_img=bg_img)
    _need(offset, "offset", 2 * _pixels(desc))
    _call("wt_composite_ca", ctypes.byref(desc), _dev(accum, "accum", f32), _dev(bg_img, "bg_img", f32),
          _dev(offset, "offset", f32), ctypes.c_float(dispersion), int(taps), _dev(out, "out", f32),
          _stream(stream))


def wt_build_resolve_batch_static(descs: Sequence[WtDesc], frags: Sequence[WtFrags],
                                  outs: Sequence[torch.Tensor],
                                  bgs: Optional[Sequence[Sequence[float]]] = None,
                                  stream=None) -> None:
    """wt_build_resolve for up to 64 frames in one launch without any device
    allocation (for callers that must not allocate when they submit work);
    see include/wt.h for the limits and the shared-scratch rule."""
    k = len(descs)
    if len(frags) != k or len(outs) != k or (bgs is not None and len(bgs) != k):
        raise ValueError(f"descs, frags, outs (and bgs) must have one entry per frame: {k}, {len(frags)}, "
                         f"{len(outs)}" + ("" if bgs is None else f", {len(bgs)}"))
    for dsc, fr, o in zip(descs, frags, outs):
        _check_frags(dsc, fr)
        _check_pixel_buffers(dsc, out=o)
    da = (WtDesc * max(k, 1))(*descs)
    fa = (WtFrags * max(k, 1))(*frags)
    bg = bgs if bgs is not None else [(0.5, 0.5, 0.5)] * k
    ba = (ctypes.c_float * max(3 * k, 3))(*[float(x) for b in bg for x in b])
    oa = (ctypes.c_void_p * max(k, 1))(*[_dev(o, "out", (torch.float32,)) for o in outs])
    _call("wt_build_resolve_batch_static", da, fa, ba, oa, k, _stream(stream))


def wt_absorbance(desc: WtDesc, coeff: torch.Tensor, pixel: torch.Tensor, z: torch.Tensor,
                  A_out: torch.Tensor, alpha: Optional[torch.Tensor] = None, stream=None) -> None:
    q = int(z.numel())
    _check_pixel_buffers(desc, coeff=coeff)
    for t, name in ((pixel, "pixel"), (A_out, "A_out"), (alpha, "alpha")):
        _need(t, name, q)
    _call("wt_absorbance", ctypes.byref(desc), _dev(coeff, "coeff", _COEFF_DT), int(z.numel()),
          _dev(pixel, "pixel", (torch.int32, torch.uint32)), _dev(z, "z", (torch.float32,)),
          _dev(alpha, "alpha", (torch.float32,)), _dev(A_out, "A_out", (torch.float32,)),
          _stream(stream))


def wt_bin_workspace_bytes(desc: WtDesc, n: int) -> int:
    return int(lib().wt_bin_workspace_bytes(ctypes.byref(desc), int(n)))


def wt_bin(desc: WtDesc, pixel: torch.Tensor, z: torch.Tensor, alpha: torch.Tensor,
           r: Optional[torch.Tensor] = None, g: Optional[torch.Tensor] = None,
           b: Optional[torch.Tensor] = None, out: Optional[dict] = None,
           workspace: Optional[torch.Tensor] = None, stream=None) -> dict:
    """Groups an unordered fragment stream by tile (wt_bin).  Returns a dict of
    the output tensors (pixel, z, alpha, r, g, b, tile_offsets); pass ``out``
    (same keys) and ``workspace`` (uint8, wt_bin_workspace_bytes(desc, n)) to
    reuse buffers.  The number of kept fragments is tile_offsets[-1]."""
    n = int(pixel.numel())
    dev = pixel.device
    rgb = r is not None
    if out is None:
        out = {"pixel": torch.empty(n, dtype=pixel.dtype, device=dev),
               "z": torch.empty(n, device=dev), "alpha": torch.empty(n, device=dev),
               "tile_offsets": torch.empty(wt_num_tiles(desc) + 1, dtype=torch.int64, device=dev)}
        if rgb:
            for k in ("r", "g", "b"):
                out[k] = torch.empty(n, device=dev)
    if workspace is None:
        workspace = torch.empty(max(1, wt_bin_workspace_bytes(desc, n)), dtype=torch.uint8, device=dev)
    fin = WtFrags(n, _dev(pixel, "pixel", (torch.int32, torch.uint32)), _dev(z, "z", (torch.float32,)),
                  _dev(alpha, "alpha", (torch.float32,)), _dev(r, "r", (torch.float32,)),
                  _dev(g, "g", (torch.float32,)), _dev(b, "b", (torch.float32,)), None)
    _call("wt_bin", ctypes.byref(desc), ctypes.byref(fin),
          _dev(out["pixel"], "pixel_out", (torch.int32, torch.uint32)),
          _dev(out["z"], "z_out", (torch.float32,)), _dev(out["alpha"], "alpha_out", (torch.float32,)),
          _dev(out.get("r"), "r_out", (torch.float32,)), _dev(out.get("g"), "g_out", (torch.float32,)),
          _dev(out.get("b"), "b_out", (torch.float32,)),
          _dev(out["tile_offsets"], "tile_offsets_out", (torch.int64,)),
          _dev(workspace, "workspace", (torch.uint8,)), int(workspace.numel()), _stream(stream))
    return out


def wt_raster(desc: WtDesc, cx: torch.Tensor, cy: torch.Tensor, radius: torch.Tensor, z: torch.Tensor,
              alpha: torch.Tensor, r: Optional[torch.Tensor] = None, g: Optional[torch.Tensor] = None,
              b: Optional[torch.Tensor] = None, capacity: Optional[int] = None, stream=None) -> dict:
    """Rasterises particles into an unordered fragment stream (wt_raster_count,
    then wt_raster_emit).  Reads the fragment total back to size the output
    (so it synchronises the stream), unless ``capacity`` is given.  Returns a
    dict of the fragment arrays (pixel, z, alpha[, r, g, b]) and "total"."""
    n = int(cx.numel())
    dev = cx.device
    f32 = (torch.float32,)
    pt = WtParticles(n, _dev(cx, "cx", f32), _dev(cy, "cy", f32), _dev(radius, "radius", f32),
                     _dev(z, "z", f32), _dev(alpha, "alpha", f32), _dev(r, "r", f32), _dev(g, "g", f32),
                     _dev(b, "b", f32))
    ws = torch.empty(int(lib().wt_raster_workspace_bytes(n)) // 8, dtype=torch.int64, device=dev)
    _call("wt_raster_count", ctypes.byref(desc), ctypes.byref(pt), _dev(ws, "workspace", (torch.int64,)),
          _stream(stream))
    total = int(ws[n].item()) if capacity is None else None
    cap = total if capacity is None else int(capacity)
    out = {"pixel": torch.empty(cap, dtype=torch.int32, device=dev), "z": torch.empty(cap, device=dev),
           "alpha": torch.empty(cap, device=dev)}
    if r is not None:
        for k in ("r", "g", "b"):
            out[k] = torch.empty(cap, device=dev)
    _call("wt_raster_emit", ctypes.byref(desc), ctypes.byref(pt), _dev(ws, "workspace", (torch.int64,)), cap,
          _dev(out["pixel"], "pixel", (torch.int32, torch.uint32)), _dev(out["z"], "z", f32),
          _dev(out["alpha"], "alpha", f32), _dev(out.get("r"), "r", f32), _dev(out.get("g"), "g", f32),
          _dev(out.get("b"), "b", f32), _stream(stream))
    out["total"] = ws[n]
    return out


def wt_raster_tri(desc: WtDesc, x: torch.Tensor, y: torch.Tensor, z: torch.Tensor, alpha: torch.Tensor,
                  r: Optional[torch.Tensor] = None, g: Optional[torch.Tensor] = None,
                  b: Optional[torch.Tensor] = None, capacity: Optional[int] = None, stream=None) -> dict:
    """Rasterises triangles (vertex arrays x, y, z of 3n, per-triangle alpha
    and colour) into an unordered fragment stream (wt_raster_tri_count, then
    wt_raster_tri_emit); otherwise as wt_raster."""
    n = int(alpha.numel())
    dev = alpha.device
    f32 = (torch.float32,)
    if x.numel() != 3 * n or y.numel() != 3 * n or z.numel() != 3 * n:
        raise ValueError("x, y and z hold three vertices per triangle")
    tr = WtTriangles(n, _dev(x, "x", f32), _dev(y, "y", f32), _dev(z, "z", f32), _dev(alpha, "alpha", f32),
                     _dev(r, "r", f32), _dev(g, "g", f32), _dev(b, "b", f32))
    ws = torch.empty(int(lib().wt_raster_workspace_bytes(n)) // 8, dtype=torch.int64, device=dev)
    _call("wt_raster_tri_count", ctypes.byref(desc), ctypes.byref(tr), _dev(ws, "workspace", (torch.int64,)),
          _stream(stream))
    total = int(ws[n].item()) if capacity is None else None
    cap = total if capacity is None else int(capacity)
    out = {"pixel": torch.empty(cap, dtype=torch.int32, device=dev), "z": torch.empty(cap, device=dev),
           "alpha": torch.empty(cap, device=dev)}
    if r is not None:
        for k in ("r", "g", "b"):
            out[k] = torch.empty(cap, device=dev)
    _call("wt_raster_tri_emit", ctypes.byref(desc), ctypes.byref(tr), _dev(ws, "workspace", (torch.int64,)), cap,
          _dev(out["pixel"], "pixel", (torch.int32, torch.uint32)), _dev(out["z"], "z", f32),
          _dev(out["alpha"], "alpha", f32), _dev(out.get("r"), "r", f32), _dev(out.get("g"), "g", f32),
          _dev(out.get("b"), "b", f32), _stream(stream))
    out["total"] = ws[n]
    return out


def wt_depth_bounds(desc: WtDesc, frags: WtFrags, zlo: torch.Tensor, zhi: torch.Tensor,
                    stream=None) -> None:
    _check_frags(desc, frags)
    _need(zlo, "zlo", _pixels(desc))
    _need(zhi, "zhi", _pixels(desc))
    _call("wt_depth_bounds", ctypes.byref(desc), ctypes.byref(frags),
          _dev(zlo, "zlo", (torch.float32,)), _dev(zhi, "zhi", (torch.float32,)), _stream(stream))


def wt_normalize_depth(desc: WtDesc, frags: WtFrags, zlo: torch.Tensor, zhi: torch.Tensor,
                       z_out: torch.Tensor, stream=None) -> None:
    _need(zlo, "zlo", _pixels(desc))
    _need(zhi, "zhi", _pixels(desc))
    _need(z_out, "z_out", int(frags.n))
    _call("wt_normalize_depth", ctypes.byref(desc), ctypes.byref(frags),
          _dev(zlo, "zlo", (torch.float32,)), _dev(zhi, "zhi", (torch.float32,)),
          _dev(z_out, "z_out", (torch.float32,)), _stream(stream))


def wt_backward(desc: WtDesc, frags: WtFrags, grad_out: torch.Tensor, grad_alpha: torch.Tensor,
                grad_rgb: torch.Tensor, bg: Sequence[float] = (0.5, 0.5, 0.5),
                bg_img: Optional[torch.Tensor] = None, stream=None,
                accum: Optional[torch.Tensor] = None) -> None:
    """grad_rgb is planar [3, n]; accum [P, 5], optional: the forward call's
    pixel sums from wt_build_resolve (the forward sums are then not recomputed)."""
    _check_frags(desc, frags)
    _check_pixel_buffers(desc, bg_img=bg_img, accum=accum)
    _need(grad_out, "grad_out", 4 * _pixels(desc))
    _need(grad_alpha, "grad_alpha", int(frags.n))
    _need(grad_rgb, "grad_rgb", 3 * int(frags.n))
    _call("wt_backward", ctypes.byref(desc), ctypes.byref(frags),
          _dev(bg_img, "bg_img", (torch.float32,)), _bg(bg),
          _dev(grad_out, "grad_out", (torch.float32,)), _dev(accum, "accum", (torch.float32,)),
          _dev(grad_alpha, "grad_alpha", (torch.float32,)),
          _dev(grad_rgb, "grad_rgb", (torch.float32,)), _stream(stream))


class WaveletOIT(torch.autograd.Function):
    """Differentiable composite: out [P, 4] = wt_build_resolve(fragments), with
    gradients for alpha and the colour planes from wt_backward (depth, pixel
    ids and tile offsets are not differentiated).  Arguments:
    (pixel, z, alpha, r, g, b, tile_offsets, desc, bg)."""

    @staticmethod
    def forward(ctx, pixel, z, alpha, r, g, b, tile_offsets, desc, bg=(0.5, 0.5, 0.5)):
        frags = make_frags(pixel, z, alpha, tile_offsets, r, g, b)
        out = torch.empty(desc.P, 4, device=z.device, dtype=torch.float32)
        accum = torch.empty(desc.P, 5, device=z.device, dtype=torch.float32)  # pixel sums, 20 B each
        wt_build_resolve(desc, frags, out, None, None, bg=bg, accum=accum)
        ctx.save_for_backward(pixel, z, alpha, r, g, b, tile_offsets, accum)
        ctx.desc = desc
        ctx.bg = tuple(bg)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        pixel, z, alpha, r, g, b, tile_offsets, accum = ctx.saved_tensors
        frags = make_frags(pixel, z, alpha, tile_offsets, r, g, b)
        n = z.numel()
        ga = torch.empty(n, device=z.device, dtype=torch.float32)
        gc = torch.empty(3, n, device=z.device, dtype=torch.float32)
        wt_backward(ctx.desc, frags, grad_out.contiguous().float(), ga, gc, bg=ctx.bg, accum=accum)
        return None, None, ga, gc[0], gc[1], gc[2], None, None, None


# ---------------------------------------------------------------- serving

class Server:
    """Continuous-batching server (wt_serve_* in include/wt.h).  The caller keeps
    each request's fragment tensors and output tensor alive until it is done."""

    def __init__(self, J: int = 4, coeff_dtype: int = BF16, flags: int = DEFAULT_FLAGS,
                 max_slots: int = 64, mem_cap_bytes: int = 40 << 30, step_tiles: int = 8192,
                 tile_w: int = 16, tile_h: int = 16):
        self.cfg = WtServeConfig(J, coeff_dtype, flags, tile_w, tile_h, max_slots, mem_cap_bytes,
                                 step_tiles)
        h = ctypes.c_void_p()
        _call("wt_serve_create", ctypes.byref(self.cfg), ctypes.byref(h))
        self._h = h
        self._keep = {}

    def submit(self, desc: WtDesc, frags: WtFrags, out: torch.Tensor,
               bg: Sequence[float] = (0.5, 0.5, 0.5), keep=None, stream=None) -> int:
        """Queues a frame whose inputs and output were produced on `stream`
        (default: torch's current stream)."""
        rid = ctypes.c_int64()
        _call("wt_serve_submit", self._h, ctypes.byref(desc), ctypes.byref(frags), _bg(bg),
              _dev(out, "out", (torch.float32,)), _stream(stream), ctypes.byref(rid))
        self._keep[rid.value] = (desc, frags, out, keep)
        return rid.value

    def wait(self, rid: int, timeout_us: int = 10_000_000) -> bool:
        """True when done; False on timeout."""
        st = lib().wt_serve_wait(self._h, rid, timeout_us)
        if st == 4:
            return False
        if st != 0:
            raise WtError("wt_serve_wait", st)
        return True

    def query(self, rid: int) -> WtServeInfo:
        info = WtServeInfo()
        _call("wt_serve_query", self._h, rid, ctypes.byref(info))
        return info

    def release(self, rid: int) -> None:
        _call("wt_serve_release", self._h, rid)
        self._keep.pop(rid, None)

    def stats(self):
        u, q, a = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        st = lib().wt_serve_stats(self._h, ctypes.byref(u), ctypes.byref(q), ctypes.byref(a))
        return {"used_bytes": u.value, "queued": q.value, "active": a.value, "status": st}

    def close(self) -> None:
        if self._h:
            _call("wt_serve_destroy", self._h)
            self._h = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Planner:
    """The server's admission / step-planning policy alone (host only)."""

    def __init__(self, max_slots: int, mem_cap_bytes: int, step_tiles: int):
        self._h = lib().wt_planner_create(max_slots, mem_cap_bytes, step_tiles)
        if not self._h:
            raise WtError("wt_planner_create", 1)

    def submit(self, nbytes: int, tiles: int) -> int:
        return int(lib().wt_planner_submit(self._h, nbytes, tiles))

    def admit(self):
        buf = (ctypes.c_int64 * 4096)()
        n = lib().wt_planner_admit(self._h, buf, 4096)
        return [buf[i] for i in range(min(n, 4096))]

    def plan(self):
        cap = 8192
        ids, t0, cnt = (ctypes.c_int64 * cap)(), (ctypes.c_int32 * cap)(), (ctypes.c_int32 * cap)()
        fin = (ctypes.c_int64 * cap)()
        nf = ctypes.c_int32(cap)
        n = lib().wt_planner_plan(self._h, ids, t0, cnt, cap, fin, ctypes.byref(nf))
        return ([(ids[i], t0[i], cnt[i]) for i in range(n)], [fin[i] for i in range(nf.value)])

    def release(self, rid: int) -> int:
        return int(lib().wt_planner_release(self._h, rid))

    def used(self) -> int:
        return int(lib().wt_planner_used(self._h))

    def close(self):
        if self._h:
            lib().wt_planner_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wt_get_error(stream=None) -> int:
    """Synchronises the stream; returns and clears the rejected-input count."""
    cnt = ctypes.c_int64(0)
    st = lib().wt_get_error(_stream(stream), ctypes.byref(cnt))
    if st not in (0, 3):
        raise WtError("wt_get_error", st)
    return int(cnt.value)
