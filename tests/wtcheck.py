"""Helpers shared by the GPU parity tests: run the CUDA path on a synthetic
frame and the FP64 oracle on the same inputs, and the tolerances.

Tolerances (derived from the arithmetic; see the design notes):
  * composite RGBA, FP32 storage: 1e-4 absolute.
  * absorbance A in front of a fragment, FP32: the relative error of
    v = exp(-A) equals the absolute error of A, held to
        |dA| <= 1e-5 * max(1, A) + 4 (J + 2) u S_p,   u = 2^-24,
    where S_p = sum of the pixel's steps: storing chi_00 ~ S_p in FP32 alone
    moves A by u S_p, and J+1 stored terms of size <= S_p enter each bin value.
    For S_p <= 16 this is within 1e-5 relative on v.
  * coefficients, FP32: |dc| <= 8 u (k + 1) S_p (k = fragments of the pixel,
    positive summands only).
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
import paper_2201_00094_gb300 as wt
import synth

U32 = 2.0 ** -24


def frags_of(g: synth.Frame):
    return wt.make_frags(g.pixel, g.z, g.alpha, g.tile_offsets, g.r, g.g, g.b)


def desc_of(fr: synth.Frame, J=None, dtype=wt.F32, flags=wt.DEFAULT_FLAGS):
    return wt.make_desc(fr.width, fr.height, fr.J if J is None else J, dtype, flags, fr.tile_w,
                        fr.tile_h)


def gpu_run(fr: synth.Frame, J=None, dtype=wt.F32, flags=wt.DEFAULT_FLAGS, bg=(0.5, 0.5, 0.5),
            bg_img=None, fused=False, two_step=False, totals=False):
    """Returns dict with coeff (float64 numpy), zmin, out [P,4] (and accum,
    and total when the build's per-pixel totals go to the resolve)."""
    dev = torch.device("cuda")
    g = fr.to(dev)
    d = desc_of(fr, J, dtype, flags)
    f = frags_of(g)
    C = 1 << d.J
    if dtype == wt.SE16:  # raw bytes: mantissas, then exponents
        coeff = wt.coeff_buffer(d, dev).fill_(0xAB)
    else:
        coeff = torch.full((fr.P, C), float("nan"), device=dev, dtype=wt.coeff_torch_dtype(dtype))
    zmin = torch.full((fr.P,), float("nan"), device=dev)
    out = torch.full((fr.P, 4), float("nan"), device=dev)
    bgt = None if bg_img is None else torch.as_tensor(bg_img, dtype=torch.float32, device=dev)
    res = {}
    if fused:
        wt.wt_build_resolve(d, f, out, coeff, zmin, bg=bg, bg_img=bgt)
    else:
        total = torch.full((fr.P,), float("nan"), device=dev) if totals else None
        wt.wt_build(d, f, coeff, zmin, total=total)
        if two_step:
            accum = torch.full((fr.P, 5), float("nan"), device=dev)
            wt.wt_resolve(d, f, coeff, zmin, accum, total=total)
            wt.wt_composite(d, accum, out, bg=bg, bg_img=bgt)
            res["accum"] = accum.cpu().numpy().astype(np.float64)
        else:
            wt.wt_resolve_composite(d, f, coeff, zmin, out, bg=bg, bg_img=bgt, total=total)
        if totals:
            res["total"] = total.cpu().numpy().astype(np.float64)
    res["bad"] = wt.wt_get_error()
    torch.cuda.synchronize()
    res["coeff"] = coeff.float().cpu().numpy().astype(np.float64)
    res["zmin"] = zmin.cpu().numpy()
    res["out"] = out.cpu().numpy().astype(np.float64)
    return res


def oracle_run(fr: synth.Frame, J=None, flags=wt.DEFAULT_FLAGS, bg=(0.5, 0.5, 0.5), bg_img=None):
    h = fr.numpy()
    J = fr.J if J is None else J
    rgb = (h["r"], h["g"], h["b"])
    c = oracle.build_coeffs(h["pixel"], h["z"], h["alpha"], fr.P, J)
    out, acc = oracle.resolve(h["pixel"], h["z"], h["alpha"], rgb, fr.P, J, c, flags=flags, bg=bg,
                              bg_img=bg_img)
    return dict(coeff=c, out=out, accum=acc)


def pixel_step_sums(fr: synth.Frame) -> np.ndarray:
    h = fr.numpy()
    a = -np.log1p(-np.clip(h["alpha"].astype(np.float64), 0, 1 - 2 ** -20))
    return np.bincount(h["pixel"].astype(np.int64), weights=a, minlength=fr.P)


def pixel_counts(fr: synth.Frame) -> np.ndarray:
    return np.bincount(fr.numpy()["pixel"].astype(np.int64), minlength=fr.P)


def coeff_tol(fr: synth.Frame) -> np.ndarray:
    S = pixel_step_sums(fr)
    k = pixel_counts(fr)
    return (8 * U32 * (k + 1) * S + 1e-30)[:, None]


def absorbance_tol(A_ref: np.ndarray, S: np.ndarray, J: int) -> np.ndarray:
    return 1e-5 * np.maximum(1.0, A_ref) + 4 * (J + 2) * U32 * S


def e5_words_of(coeffs, C):
    """E5B9G9R9 words of three channels' [P, C] coefficients, encoded by the
    oracle (the stored magnitudes are chi_00 and -X_{n,k}, §2.3.1)."""
    sign = np.where(np.arange(C) == 0, 1.0, -1.0).astype(np.float32)
    return oracle.e5_encode(*[np.asarray(c, np.float32) * sign for c in coeffs])


def e5_oracle_composite(h, alphas, P, J, bg, words_gpu, flags=None, bg_img=None):
    """The E5B9G9R9 composite computed wholly on the oracle side -- FP64
    coefficients rounded to FP32, encoded and decoded by the oracle -- and the
    per-pixel bound within which the GPU's must lie.  The GPU's FP32
    coefficients can round across a mantissa tie differently from FP64's in
    rare last places; at a pixel whose words differ, each differing index i
    (level n) moves a bin value by at most 2^(n/2) times the mantissa steps
    of the two words, and the composite is 1-Lipschitz in the absorbance
    (the normalised colour moves by at most tanh of it).  `flags` selects the
    reading (default: the method's), `bg_img` [P, 3] a background image.
    Returns (reference, bound per pixel, words equal per pixel)."""
    C = 1 << J
    sign = np.where(np.arange(C) == 0, 1.0, -1.0)
    co = [oracle.build_coeffs(h["pixel"], h["z"], alphas[c], P, J).astype(np.float32) for c in range(3)]
    w = e5_words_of(co, C)
    dec = oracle.e5_decode(w)
    flags = oracle.DEFAULT_FLAGS if flags is None else flags
    if bg_img is None:
        ref = oracle.composite_rgb(h["pixel"], h["z"], alphas, (h["r"], h["g"], h["b"]), P, J, flags=flags,
                                   bg=bg, coeffs=[sign * dec[c] for c in range(3)])
    else:
        ref = np.zeros((P, 4))
        for c in range(3):
            col = (h["r"], h["g"], h["b"])[c]
            bgc = np.repeat(np.asarray(bg_img)[:, c:c + 1], 3, axis=1)
            o = oracle.resolve(h["pixel"], h["z"], alphas[c], (col,) * 3, P, J, sign * dec[c], flags,
                               bg_img=bgc)[0]
            ref[:, c] = o[:, 0]
            ref[:, 3] += o[:, 3] / 3.0
    lvl = np.array([0] + [int(np.log2(i)) for i in range(1, C)])
    step = lambda x: np.ldexp(1.0, (x >> 27).astype(np.int64) - 24)
    diff = w != words_gpu
    bound = 1e-4 + (diff * np.sqrt(2.0) ** lvl * (step(w) + step(words_gpu))).sum(axis=1)
    return ref, bound, ~diff.any(axis=1)
