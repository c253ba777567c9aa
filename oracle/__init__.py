"""FP64 CPU oracle for Wavelet Transparency (paper §2), reached through ctypes.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its binding) never imports this package, and this package
imports nothing from the product.

The C source (``wt_oracle.c``) is compiled on first use with gcc into
``liboracle.so`` beside it; ``build()`` does the same eagerly.
"""
from __future__ import annotations

import ctypes
import fcntl
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wt_oracle.c")
_HDR = os.path.join(_HERE, "wt_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")

# reading flags (the oracle's own definitions; numerically equal to the library's)
SELF_EXCLUDE = 1
INTERP_LINEAR = 2
RESOLVE_NORMALIZED = 4
DEFAULT_FLAGS = SELF_EXCLUDE | INTERP_LINEAR | RESOLVE_NORMALIZED

_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so (plain C11, -O2, no OpenMP: single-threaded)."""
    lock = _LIB + ".lock"
    with open(lock, "w") as lf:
        fcntl.flock(lf, fcntl.LOCK_EX)
        stale = not os.path.exists(_LIB) or any(
            os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    P = ctypes.c_void_p
    i64, i32, u32 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint32
    lib.wto_psi.argtypes = [i32, i32, ctypes.c_double]
    lib.wto_psi.restype = ctypes.c_double
    lib.wto_Psi.argtypes = [i32, i32, ctypes.c_double]
    lib.wto_Psi.restype = ctypes.c_double
    lib.wto_build.argtypes = [i64, P, P, P, i64, i32, P]
    lib.wto_build_binned.argtypes = [i64, P, P, P, i64, i32, P]
    lib.wto_bin_values.argtypes = [P, i32, P]
    lib.wto_bin_values.restype = None
    lib.wto_recon.argtypes = [P, i32, ctypes.c_double, i32]
    lib.wto_recon.restype = ctypes.c_double
    lib.wto_fragment_absorbance.argtypes = [i64, P, P, P, i64, i32, u32, P, P]
    lib.wto_absorbance_at.argtypes = [i64, P, P, i64, i32, u32, P, P]
    lib.wto_resolve.argtypes = [i64, P, P, P, P, P, P, i64, i32, u32, P, P, P, P, P]
    lib.wto_abuffer.argtypes = [i64, P, P, P, P, P, P, i64, P, P, P]
    lib.wto_grad.argtypes = [i64, P, P, P, P, P, P, i64, i32, u32, P, P, P, P, P]
    lib.wto_depth_bounds.argtypes = [i64, P, P, P, i64, P, P]
    lib.wto_normalize_depth.argtypes = [i64, P, P, i64, P, P, P]
    for f in ("wto_build", "wto_build_binned", "wto_fragment_absorbance", "wto_absorbance_at",
              "wto_resolve", "wto_abuffer", "wto_grad"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _u32(a):
    return np.ascontiguousarray(np.asarray(a), dtype=np.uint32)


def _f32(a):
    return np.ascontiguousarray(np.asarray(a), dtype=np.float32)


def _f64(a):
    return None if a is None else np.ascontiguousarray(np.asarray(a), dtype=np.float64)


def _check(st, name):
    if st != 0:
        raise ValueError(f"oracle {name} failed with status {st}")


def psi(n: int, k: int, x: float) -> float:
    return _load().wto_psi(n, k, x)


def Psi(n: int, k: int, x: float) -> float:
    return _load().wto_Psi(n, k, x)


def build_coeffs(pixel, z, alpha, P: int, J: int) -> np.ndarray:
    """Closed-form coefficients (§2.3.1) -> float64 [P, 2^J]."""
    pixel, z, alpha = _u32(pixel), _f32(z), _f32(alpha)
    out = np.zeros((P, 1 << J), np.float64)
    _check(_load().wto_build(len(z), _ptr(pixel), _ptr(z), _ptr(alpha), P, J, _ptr(out)), "build")
    return out


def build_coeffs_binned(pixel, z, alpha, P: int, J: int) -> np.ndarray:
    """Independent construction: exact bin averages + Haar analysis."""
    pixel, z, alpha = _u32(pixel), _f32(z), _f32(alpha)
    out = np.zeros((P, 1 << J), np.float64)
    _check(_load().wto_build_binned(len(z), _ptr(pixel), _ptr(z), _ptr(alpha), P, J, _ptr(out)),
           "build_binned")
    return out


def bin_values(coeff_row, J: int) -> np.ndarray:
    c = _f64(coeff_row)
    out = np.zeros(1 << J, np.float64)
    _load().wto_bin_values(_ptr(c), J, _ptr(out))
    return out


def recon(abar, J: int, x: float, linear: bool = True) -> float:
    a = _f64(abar)
    return _load().wto_recon(_ptr(a), J, float(x), int(linear))


def fragment_absorbance(pixel, z, alpha, P, J, coeff, flags=DEFAULT_FLAGS) -> np.ndarray:
    pixel, z, alpha, coeff = _u32(pixel), _f32(z), _f32(alpha), _f64(coeff)
    out = np.zeros(len(z), np.float64)
    _check(_load().wto_fragment_absorbance(len(z), _ptr(pixel), _ptr(z), _ptr(alpha), P, J,
                                           flags, _ptr(coeff), _ptr(out)), "fragment_absorbance")
    return out


def absorbance_at(pixel, z, P, J, coeff, flags=DEFAULT_FLAGS) -> np.ndarray:
    pixel, z, coeff = _u32(pixel), _f32(z), _f64(coeff)
    out = np.zeros(len(z), np.float64)
    _check(_load().wto_absorbance_at(len(z), _ptr(pixel), _ptr(z), P, J, flags, _ptr(coeff),
                                     _ptr(out)), "absorbance_at")
    return out


def resolve(pixel, z, alpha, rgb, P, J, coeff, flags=DEFAULT_FLAGS, bg=(0.5, 0.5, 0.5),
            bg_img=None):
    """Resolve + composite.  rgb is [n,3] or a tuple (r, g, b).

    Returns (out [P,4], accum [P,6] = {R',G',B',W',S,Amin})."""
    pixel, z, alpha, coeff = _u32(pixel), _f32(z), _f32(alpha), _f64(coeff)
    r, g, b = _split_rgb(rgb)
    out = np.zeros((P, 4), np.float64)
    acc = np.zeros((P, 6), np.float64)
    bgv = _f64(bg)
    _check(_load().wto_resolve(len(z), _ptr(pixel), _ptr(z), _ptr(alpha), _ptr(r), _ptr(g),
                               _ptr(b), P, J, flags, _ptr(coeff), _ptr(bgv), _ptr(_f64(bg_img)),
                               _ptr(acc), _ptr(out)), "resolve")
    return out, acc


def composite(pixel, z, alpha, rgb, P, J, flags=DEFAULT_FLAGS, bg=(0.5, 0.5, 0.5), bg_img=None):
    """Build + resolve + composite in one call -> out [P,4]."""
    coeff = build_coeffs(pixel, z, alpha, P, J)
    return resolve(pixel, z, alpha, rgb, P, J, coeff, flags, bg, bg_img)[0]


def abuffer(pixel, z, alpha, rgb, P, bg=(0.5, 0.5, 0.5), bg_img=None) -> np.ndarray:
    """Exact sorted front-to-back composite -> out [P,4]."""
    pixel, z, alpha = _u32(pixel), _f32(z), _f32(alpha)
    r, g, b = _split_rgb(rgb)
    out = np.zeros((P, 4), np.float64)
    _check(_load().wto_abuffer(len(z), _ptr(pixel), _ptr(z), _ptr(alpha), _ptr(r), _ptr(g),
                               _ptr(b), P, _ptr(_f64(bg)), _ptr(_f64(bg_img)), _ptr(out)),
           "abuffer")
    return out


def grad(pixel, z, alpha, rgb, P, J, gout, flags=DEFAULT_FLAGS, bg=(0.5, 0.5, 0.5), bg_img=None):
    """Analytic gradient of sum(gout * out) -> (d alpha [n], d rgb [n,3])."""
    pixel, z, alpha = _u32(pixel), _f32(z), _f32(alpha)
    r, g, b = _split_rgb(rgb)
    n = len(z)
    ga = np.zeros(n, np.float64)
    gc = np.zeros((n, 3), np.float64)
    go = _f64(gout).reshape(P, 4)
    _check(_load().wto_grad(n, _ptr(pixel), _ptr(z), _ptr(alpha), _ptr(r), _ptr(g), _ptr(b), P,
                            J, flags, _ptr(_f64(bg)), _ptr(_f64(bg_img)), _ptr(go), _ptr(ga),
                            _ptr(gc)), "grad")
    return ga, gc


def _split_rgb(rgb):
    if isinstance(rgb, (tuple, list)) and len(rgb) == 3:
        return tuple(_f32(c) for c in rgb)
    a = np.asarray(rgb, dtype=np.float32)
    return _f32(a[:, 0]), _f32(a[:, 1]), _f32(a[:, 2])


def depth_bounds(pixel, z, alpha, P: int):
    """Per-pixel (min, max) depth of the pixel's fragments (§2.1 step 1)."""
    pixel, z, alpha = _u32(pixel), _f32(z), _f32(alpha)
    lo, hi = np.empty(P), np.empty(P)
    _check(_load().wto_depth_bounds(len(pixel), _ptr(pixel), _ptr(z), _ptr(alpha), P, _ptr(lo), _ptr(hi)),
           "wto_depth_bounds")
    return lo, hi


def normalize_depth(pixel, z, P: int, zlo, zhi) -> np.ndarray:
    """Depth mapped into its pixel's bounds, (z - lo) / (hi - lo)."""
    pixel, z = _u32(pixel), _f32(z)
    zlo, zhi = _f64(zlo), _f64(zhi)
    out = np.empty(len(pixel))
    _check(_load().wto_normalize_depth(len(pixel), _ptr(pixel), _ptr(z), P, _ptr(zlo), _ptr(zhi), _ptr(out)),
           "wto_normalize_depth")
    return out


def tile_of_pixels(pixel, width: int, height: int, tile_w: int, tile_h: int) -> np.ndarray:
    """Row-major tile id of each pixel id (y * width + x); -1 outside the image."""
    pixel = np.asarray(pixel, dtype=np.int64)
    ntx = -(-width // tile_w)
    y, x = pixel // width, pixel % width
    t = (y // tile_h) * ntx + x // tile_w
    return np.where(pixel < width * height, t, -1)


def bin_by_tile(pixel, width: int, height: int, tile_w: int, tile_h: int):
    """Fragments grouped by tile: a stable counting sort by tile id (the
    library sort stands in for the counting).  Returns (order, tile_offsets):
    kept fragment indices in tile order, and [ntiles + 1] offsets; fragments
    outside the image are dropped."""
    t = tile_of_pixels(pixel, width, height, tile_w, tile_h)
    ntiles = -(-width // tile_w) * -(-height // tile_h)
    keep = np.nonzero(t >= 0)[0]
    order = keep[np.argsort(t[keep], kind="stable")]
    counts = np.bincount(t[keep], minlength=ntiles)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return order, offsets


def raster_particles(width: int, height: int, cx, cy, radius, z, alpha, r=None, g=None, b=None):
    """Fragments of screen-space disc particles, in particle order and
    row-major inside a particle: a fragment on every pixel whose centre
    (x + 1/2, y + 1/2) is at squared distance d2 < radius^2 from the centre,
    opacity alpha * (1 - d2 * (1 / radius^2)).  Every operation is one FP32
    operation rounded to nearest (the coverage decision is taken in FP32, the
    precision of the definition).  Plain loops over particles and rows."""
    f = np.float32
    cx, cy, radius, z, alpha = (np.asarray(v, dtype=f) for v in (cx, cy, radius, z, alpha))
    cols = {"pixel": [], "z": [], "alpha": []}
    rgb = r is not None
    if rgb:
        r, g, b = (np.asarray(v, dtype=f) for v in (r, g, b))
        cols.update(r=[], g=[], b=[])
    for i in range(len(cx)):
        rho = radius[i]
        if not (rho > 0) or np.isnan(cx[i]) or np.isnan(cy[i]) or not (rho < 1e6) \
                or not (abs(cx[i]) < 1e9) or not (abs(cy[i]) < 1e9):
            continue
        rho2 = f(rho * rho)
        inv = f(f(1) / rho2)
        x0 = max(0, int(np.floor(float(cx[i]) - float(rho))) - 2)
        x1 = min(width - 1, int(np.ceil(float(cx[i]) + float(rho))) + 2)
        y0 = max(0, int(np.floor(float(cy[i]) - float(rho))) - 2)
        y1 = min(height - 1, int(np.ceil(float(cy[i]) + float(rho))) + 2)
        if x1 < x0 or y1 < y0:
            continue
        xs = np.arange(x0, x1 + 1)
        dx = (xs.astype(f) + f(0.5)) - cx[i]
        dx2 = dx * dx
        for y in range(y0, y1 + 1):
            dy = f(f(y) + f(0.5)) - cy[i]
            d2 = dx2 + f(dy * dy)
            hit = d2 < rho2
            if not hit.any():
                continue
            cols["pixel"].append((y * width + xs[hit]).astype(np.int64))
            cols["alpha"].append(alpha[i] * (f(1) - d2[hit] * inv))
            cols["z"].append(np.full(hit.sum(), z[i], dtype=f))
            if rgb:
                for k, v in (("r", r), ("g", g), ("b", b)):
                    cols[k].append(np.full(hit.sum(), v[i], dtype=f))
    out = {}
    for k, v in cols.items():
        dt = np.int64 if k == "pixel" else f
        out[k] = np.concatenate(v).astype(dt) if v else np.zeros(0, dtype=dt)
    return out


def raster_triangles(width: int, height: int, x, y, z, alpha, r=None, g=None, b=None):
    """Fragments of screen-space triangles (glass panes: two per quad), in
    triangle order and row-major inside a triangle.  Vertex k of triangle i is
    (x, y, z)[3i + k]; opacity and colour are per triangle.

    Coverage is decided exactly: the vertices are snapped to 1/256 pixel,
    X = rint(256 x), and pixel (px, py) is covered when its centre
    C = (256 px + 128, 256 py + 128) is inside, with the edge functions in
    integers, E(A->B) = (Bx - Ax)(Cy - Ay) - (By - Ay)(Cx - Ax), on the
    triangle wound so that its area E(v0->v1)(v2) is positive: every E > 0, or
    E = 0 on an edge with dy < 0, or dy = 0 and dx > 0 (the edge the centre
    would enter when moved right and infinitesimally down, so that a centre on
    an edge or vertex shared by triangles that tile the plane belongs to
    exactly one of them).  Zero-area triangles, non-finite vertices and vertices
    at |x| or |y| >= 2^22 give no fragments.  Depth at the centre from the
    barycentric weights e_k = float32(E_k) opposite vertex k:
    z = ((e0 z0 + e1 z1) + e2 z2) / float32(area), each operation one FP32
    rounding."""
    f = np.float32
    x, y, z, alpha = (np.asarray(v, dtype=f) for v in (x, y, z, alpha))
    cols = {"pixel": [], "z": [], "alpha": []}
    rgb = r is not None
    if rgb:
        r, g, b = (np.asarray(v, dtype=f) for v in (r, g, b))
        cols.update(r=[], g=[], b=[])
    lim = f(4194304.0)  # 2^22
    for i in range(len(alpha)):
        vx, vy, vz = x[3 * i:3 * i + 3], y[3 * i:3 * i + 3], z[3 * i:3 * i + 3].copy()
        if not (np.all(np.abs(vx) < lim) and np.all(np.abs(vy) < lim)):
            continue  # also rejects NaN
        X = [int(np.rint(v * f(256))) for v in vx]
        Y = [int(np.rint(v * f(256))) for v in vy]
        area = (X[1] - X[0]) * (Y[2] - Y[0]) - (Y[1] - Y[0]) * (X[2] - X[0])
        if area == 0:
            continue
        if area < 0:
            X[1], X[2] = X[2], X[1]
            Y[1], Y[2] = Y[2], Y[1]
            vz[1], vz[2] = vz[2], vz[1]
            area = -area
        x0 = max(0, (min(X) - 128) // 256)
        x1 = min(width - 1, (max(X) - 128) // 256 + 1)
        y0 = max(0, (min(Y) - 128) // 256)
        y1 = min(height - 1, (max(Y) - 128) // 256 + 1)
        if x1 < x0 or y1 < y0:
            continue
        edges = [(1, 2), (2, 0), (0, 1)]  # edge k is opposite vertex k
        for py in range(y0, y1 + 1):
            cy = 256 * py + 128
            for px in range(x0, x1 + 1):
                cx = 256 * px + 128
                E = []
                inside = True
                for a_, b_ in edges:
                    dx, dy = X[b_] - X[a_], Y[b_] - Y[a_]
                    e = dx * (cy - Y[a_]) - dy * (cx - X[a_])
                    if e < 0 or (e == 0 and not (dy < 0 or (dy == 0 and dx > 0))):
                        inside = False
                        break
                    E.append(e)
                if not inside:
                    continue
                e0, e1, e2 = (f(v) for v in E)
                zz = f(f(f(e0 * vz[0]) + f(e1 * vz[1])) + f(e2 * vz[2])) / f(area)
                cols["pixel"].append(np.array([py * width + px], dtype=np.int64))
                cols["z"].append(np.array([zz], dtype=f))
                cols["alpha"].append(np.array([alpha[i]], dtype=f))
                if rgb:
                    for k, v in (("r", r), ("g", g), ("b", b)):
                        cols[k].append(np.array([v[i]], dtype=f))
    out = {}
    for k, v in cols.items():
        dt = np.int64 if k == "pixel" else f
        out[k] = np.concatenate(v).astype(dt) if v else np.zeros(0, dtype=dt)
    return out


def composite_rgb(pixel, z, alpha_c, rgb, P: int, J: int, flags=DEFAULT_FLAGS, bg=(0.5, 0.5, 0.5),
                  coeffs=None) -> np.ndarray:
    """Coloured absorbance: channel c is the mono method with its own opacity
    alpha_c[c] and its own colour component rgb[c] (§1.2, §2.1); out[:, c] is
    its composite and out[:, 3] the mean of the three coverages 1 - T_c.
    `coeffs` (three [P, C] arrays) replaces the channels' own coefficients."""
    out = np.zeros((P, 4))
    for c in range(3):
        co = build_coeffs(pixel, z, alpha_c[c], P, J) if coeffs is None else coeffs[c]
        o = resolve(pixel, z, alpha_c[c], (rgb[c], rgb[c], rgb[c]), P, J, co, flags, (bg[c],) * 3)[0]
        out[:, c] = o[:, 0]
        out[:, 3] += o[:, 3] / 3.0
    return out


def e5_encode(r, g, b) -> np.ndarray:
    """E5B9G9R9 words of three non-negative arrays (§2.1: the coefficients of
    the three channels are packed into 32 bits with a shared exponent; the bit
    layout is the shared-exponent format the name denotes: 9-bit mantissas,
    5-bit exponent, bias 15).  Values are
    clamped to [0, 511/512 * 2^16]; the exponent comes from the largest channel,
    floor(log2(max)) + 16 (at least 0), raised by one if that channel's rounded
    mantissa reaches 512; mantissas are floor(v / 2^(e - 24) + 1/2).  Every
    step is one FP32 operation, as in the definition's integer decisions."""
    f = np.float32
    r, g, b = (np.clip(np.nan_to_num(np.asarray(v, dtype=f), nan=0.0), f(0), f(65408.0)).astype(f)
               for v in (r, g, b))
    mx = np.maximum(r, np.maximum(g, b))
    expo = ((mx.view(np.uint32) >> 23) & 0xFF).astype(np.int64) - 127
    fl = np.where(mx > 0, np.maximum(expo, -16), -16)
    e = fl + 16
    scale = np.ldexp(np.ones_like(mx), 24 - e).astype(f)
    bump = np.floor(mx * scale + f(0.5)) >= 512
    e = np.where(bump, e + 1, e)
    scale = np.where(bump, scale * f(0.5), scale).astype(f)
    q = [np.floor(v * scale + f(0.5)).astype(np.uint64) for v in (r, g, b)]
    return (q[0] | (q[1] << 9) | (q[2] << 18) | (e.astype(np.uint64) << 27)).astype(np.uint32)


def e5_decode(w):
    """The three values of E5B9G9R9 words: mantissa * 2^(e - 24)."""
    w = np.asarray(w, dtype=np.uint32).astype(np.uint64)
    scale = np.ldexp(1.0, (w >> 27).astype(np.int64) - 24)
    return tuple((((w >> s) & 511).astype(np.float64) * scale) for s in (0, 9, 18))


# ---------------------------------------------------------------- shared-exponent 16-bit storage

SE16_EMIN, SE16_EMAX, SE16_BIAS = -100, 100, 128


def se16_level_shift(J: int) -> np.ndarray:
    """floor(n / 2) for every heap index of a row of 2^J coefficients (0 for
    chi_00; index 2^n + k is on level n)."""
    C = 1 << J
    sh = np.zeros(C, np.int64)
    for i in range(1, C):
        sh[i] = (i.bit_length() - 1) // 2
    return sh


def se16_encode(coeff, J: int):
    """Mono coefficients [P, 2^J] -> (mantissas uint16 [P, 2^J], exponent
    bytes uint8 [P]), the 16-bit shared-exponent storage.

    The format rests on the sign property of §2.3.1 (chi_00 >= 0, every
    X_{n,k} <= 0), which lets every coefficient be stored as an unsigned
    magnitude, as the paper does for its E5B9G9R9 words (§2.1); here the
    exponent is shared by the 2^J coefficients of one pixel instead of the
    three channels of one coefficient.  Per pixel:
      m_0 = chi_00, m_i = -X_{n,k} 2^floor(n/2)  (i = 2^n + k; both clamped
            at 0, NaN -> 0; the power of two keeps every m_i <= sum of the
            pixel's steps, since |X_{n,k}| <= 2^(-n/2) S / 2);
      M = max_i m_i;  e = floor(log2 M) + 1 from M's FP32 exponent, clamped
            to [-100, 100] (e = -100 when M is 0 or below 2^-126);
      q_i = rint(m_i 2^(16 - e)) (half to even); if the largest q reaches
            2^16, e is raised by one and the q_i taken again;
      exponent byte = e + 128.
    Every product and rounding is one FP32 operation, so the integer codes
    are those of the definition applied to the given FP32 values."""
    f = np.float32
    c = np.asarray(coeff, dtype=f)
    P, C = c.shape
    assert C == 1 << J
    sh = se16_level_shift(J)
    neg = np.concatenate([np.ones(1, f), -np.ones(C - 1, f)])
    m = np.fmax(c * neg, f(0)) * np.ldexp(f(1), sh).astype(f)  # exact scalings
    M = m.max(axis=1)
    bits = M.view(np.uint32)
    ex = ((bits >> 23) & 0xFF).astype(np.int64)
    e = np.where(ex > 0, ex - 127 + 1, SE16_EMIN)
    e = np.clip(e, SE16_EMIN, SE16_EMAX)

    def quant(e):
        scale = np.ldexp(f(1), 16 - e).astype(f)
        return np.rint(m * scale[:, None]).astype(f)

    q = quant(e)
    bump = q.max(axis=1) >= 65536
    e = np.where(bump, e + 1, e)
    q = np.where(bump[:, None], quant(e), q)
    q = np.minimum(q, 65535)
    return q.astype(np.uint16), (e + SE16_BIAS).astype(np.uint8)


def se16_decode(mant, expo, J: int) -> np.ndarray:
    """Coefficients [P, 2^J] (float64) of shared-exponent 16-bit rows:
    chi_00 = q_0 2^(e - 16), X_{n,k} = -q_i 2^(e - 16 - floor(n/2))."""
    q = np.asarray(mant, dtype=np.uint16).astype(np.float64)
    e = np.asarray(expo, dtype=np.uint8).astype(np.int64) - SE16_BIAS
    sh = se16_level_shift(J)
    sign = np.concatenate([np.ones(1), -np.ones((1 << J) - 1)])
    return sign * q * np.ldexp(1.0, e[:, None] - 16 - sh[None, :])


def se16_split(buf, P: int, J: int):
    """(mantissas [P, 2^J], exponent bytes [P]) of a storage buffer in the
    library's layout: P * 2^J little-endian uint16 mantissas, pixel-major in
    heap order, followed by P exponent bytes."""
    raw = np.asarray(buf).view(np.uint8).reshape(-1)
    C = 1 << J
    mant = raw[:2 * P * C].view(np.uint16).reshape(P, C)
    expo = raw[2 * P * C:2 * P * C + P]
    return mant, expo


# ---------------------------------------------------------------- chromatic aberration (§3)

def _smoothstep(e0: float, e1: float, x):
    """GLSL smoothstep written out: u = clamp((x - e0) / (e1 - e0), 0, 1),
    u^2 (3 - 2u).  The formula is applied as written also when e0 > e1, as the
    §3 listing does (the result then falls from 1 to 0)."""
    u = np.clip((np.asarray(x, dtype=np.float64) - e0) / (e1 - e0), 0.0, 1.0)
    return u * u * (3.0 - 2.0 * u)


def spectral_weights(taps: int) -> np.ndarray:
    """[taps, 3] colour weights of the chromatic-aberration gather (§3).  Tap i
    sits at t_i = i / (taps - 1) along the segment (the listing's printed
    t = 1/2 + 2i/(k-1) leaves [0, 1] after the first tap, so the taps are read as
    spread evenly over [0, 1]); w_r = smoothstep(1/2, 1/3, t),
    w_b = smoothstep(1/2, 2/3, t), w_g = 1 - w_r - w_b.  One tap: weight 1."""
    if taps == 1:
        return np.ones((1, 3))
    t = np.arange(taps) / (taps - 1)
    wr = _smoothstep(0.5, 1.0 / 3.0, t)
    wb = _smoothstep(0.5, 2.0 / 3.0, t)
    return np.stack([wr, 1.0 - wr - wb, wb], axis=1)


def tap_scales(taps: int, dispersion: float) -> np.ndarray:
    """Positions of the taps along the refraction offset d, as multiples of d:
    a segment centred on the refracted sample point p + d, of length
    dispersion * |d| (proportional to the refraction, §3): s_i = 1 +
    dispersion (t_i - 1/2)."""
    if taps == 1:
        return np.ones(1)
    t = np.arange(taps) / (taps - 1)
    return 1.0 + dispersion * (t - 0.5)


def bilinear(img, width: int, height: int, x, y) -> np.ndarray:
    """Bilinear sample of an RGB image [P, 3] at continuous pixel positions
    (x, y) (texel (i, j) centred at (i + 1/2, j + 1/2)), clamped to the edge."""
    img = np.asarray(img, dtype=np.float64).reshape(height * width, 3)
    fx, fy = np.asarray(x, dtype=np.float64) - 0.5, np.asarray(y, dtype=np.float64) - 0.5
    x0, y0 = np.floor(fx), np.floor(fy)
    ax, ay = (fx - x0)[..., None], (fy - y0)[..., None]
    i0 = np.clip(x0, 0, width - 1).astype(np.int64)
    i1 = np.clip(x0 + 1, 0, width - 1).astype(np.int64)
    j0 = np.clip(y0, 0, height - 1).astype(np.int64)
    j1 = np.clip(y0 + 1, 0, height - 1).astype(np.int64)
    s = lambda i, j: img[j * width + i]
    return ((1 - ax) * (1 - ay) * s(i0, j0) + ax * (1 - ay) * s(i1, j0)
            + (1 - ax) * ay * s(i0, j1) + ax * ay * s(i1, j1))


def ca_background(bg_img, offset, width: int, height: int, dispersion: float, taps: int,
                  pixels=None) -> np.ndarray:
    """The background seen through the transparent layers with chromatic
    aberration (§3): instead of one bilinear sample at the refracted point
    p + d, `taps` samples along the segment of tap_scales, each channel the
    weighted mean of the samples under its spectral weight.  A pixel whose
    offset is not finite takes the unshifted background.  `pixels` (ids)
    restricts the result to those pixels."""
    P = width * height
    px = np.arange(P) if pixels is None else np.asarray(pixels, dtype=np.int64)
    d = np.asarray(offset, dtype=np.float64).reshape(P, 2)[px].copy()
    bad = ~np.isfinite(d).all(axis=1)
    d[bad] = 0.0
    x, y = px % width + 0.5, px // width + 0.5
    w = spectral_weights(taps)
    acc = np.zeros((len(px), 3))
    for i, s in enumerate(tap_scales(taps, dispersion)):
        acc += w[i] * bilinear(bg_img, width, height, x + s * d[:, 0], y + s * d[:, 1])
    return acc / w.sum(axis=0)


def composite_ca(accum, bg_img, offset, width: int, height: int, dispersion: float = 0.5, taps: int = 5,
                 flags=DEFAULT_FLAGS, pixels=None) -> np.ndarray:
    """§2.1 step 4 with the chromatic-aberration background of §3: the
    composite of `resolve`'s accumulators (accum [P, 6] = R', G', B', W', S, Amin)
    over ca_background instead of the background pixel.  With `pixels`, accum
    holds those pixels' rows only."""
    a = np.asarray(accum, dtype=np.float64)
    bgc = ca_background(bg_img, offset, width, height, dispersion, taps, pixels)
    R, W, S, Amin = a[:, :3], a[:, 3:4], a[:, 4:5], a[:, 5:6]
    T = np.exp(-S)
    out = np.zeros((a.shape[0], 4))
    if flags & RESOLVE_NORMALIZED:
        with np.errstate(divide="ignore", invalid="ignore"):
            out[:, :3] = np.where(W > 0, R / np.where(W > 0, W, 1.0) * (1.0 - T) + bgc * T, bgc)
    else:
        out[:, :3] = R * np.exp(-Amin) + bgc * T
    out[:, 3] = 1.0 - T[:, 0]
    return out
