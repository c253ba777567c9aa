/*
 * wt.h -- C ABI of the GB300 Wavelet OIT library (libwt.so).
 *
 * The library implements the hot path of "Wavelet Transparency"
 * (Aizenshtein, Smal & McGuire, 2021) as hand-written CUDA for sm_103a:
 *
 *   build    (§2.1 step 2, §2.3.1)  project every fragment's absorbance step
 *            a = -ln(1 - alpha) at normalised depth z onto a per-pixel Haar
 *            basis of C = 2^J coefficients;
 *   resolve  (§2.1 step 3, §2.2, §2.3.2)  reconstruct A(z) at each fragment,
 *            v = exp(-A), and accumulate the order-independent weighted colour;
 *   composite (§2.1 step 4)  composite the accumulation over the background.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - All array arguments are DEVICE pointers owned by the caller (for example
 *   torch tensors).  The library never allocates, frees or retains them.
 * - Every call is asynchronous on the given stream (NULL = legacy default
 *   stream) and returns after the launch.  Argument errors are detected on the
 *   host and returned synchronously; nothing is launched in that case.
 * - Data errors (a fragment whose pixel id is >= width*height or lies outside
 *   the tile it is filed under, NaN z or alpha, a decreasing tile_offsets
 *   pair) are never fatal: the fragment (or tile range) is skipped and counted
 *   in a per-device error word that wt_get_error() reads and clears.  No kernel
 *   traps, asserts or spins.
 * - Pixel id = y * width + x.  Coefficients are pixel-major,
 *   coeff[p * C + j], in heap order: j = 0 holds chi_00, j = 2^n + k holds
 *   X_{n,k} for level n = 0..J-1 and shift k = 0..2^n-1 (§2.3).
 * - Depth is normalised to [0, 1) (the per-pixel bounds of §2.1 step 1 are
 *   applied before the build, e.g. with wt_depth_bounds and
 *   wt_normalize_depth); z is clamped to [0, 1 - 2^-24] and alpha to
 *   [0, 1 - 2^-20] before use.
 * - The build, resolve and composite calls take a stream grouped by screen
 *   tile (wt_frags.tile_offsets); wt_bin groups an unordered stream.
 * - Float pointers must be 16-byte aligned.
 */
#ifndef WT_H
#define WT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; declared here so that the header needs no CUDA
 * include. */
typedef struct CUstream_st *wt_stream;

typedef enum wt_status {
    WT_OK = 0,
    WT_ERR_ARG = 1,         /* bad argument: NULL, size out of range, misaligned */
    WT_ERR_UNSUPPORTED = 2, /* valid but not supported (J > 6, a J and tile size whose
                               shared memory exceeds one CTA's, flag combination) */
    WT_ERR_INPUT = 3,       /* reported by wt_get_error when fragments were rejected */
    WT_ERR_TIMEOUT = 4,     /* a bounded wait ran out (serving) */
    WT_ERR_CUDA = 5,        /* a CUDA runtime call failed (launch error, bad device) */
    WT_ERR_NOMEM = 6,       /* a request exceeds a memory cap (serving) */
    WT_ERR_BUSY = 7         /* no free slot (serving) */
} wt_status;

/* Storage type of the coefficient buffer; accumulation is always FP32.
 *
 * WT_SE16 is 16-bit storage with a shared exponent per pixel, resting on the
 * sign property of §2.3.1 (chi_00 >= 0 and every X_{n,k} <= 0, so every
 * coefficient is stored as a magnitude, as §2.1 does for its E5B9G9R9 words).
 * For each pixel, with i = 2^n + k the heap index of X_{n,k}:
 *     m_0 = chi_00,  m_i = -X_{n,k} * 2^floor(n/2)   (each clamped at 0);
 *     e   = floor(log2(max_i m_i)) + 1, clamped to [-100, 100];
 *     q_i = rint(m_i * 2^(16 - e)) (ties to even), unsigned 16-bit; if the
 *           largest q_i reaches 2^16, e is raised by one and the q_i retaken.
 * The buffer holds the q_i as uint16 [P][C] (pixel-major, heap order, where a
 * BF16 row would be), followed by P exponent bytes (e + 128).  A stored value
 * decodes to chi_00 = q_0 2^(e-16), X_{n,k} = -q_i 2^(e-16-floor(n/2)), and is
 * within half a unit of 2^(e-16) of the FP32 value: the error is set by the
 * pixel's largest magnitude (at most its total step), not by each
 * coefficient's own size, which is what keeps deep pixels accurate where
 * BF16's 8-bit significand does not. */
typedef enum wt_dtype { WT_F32 = 0, WT_BF16 = 1, WT_F16 = 2, WT_SE16 = 3 } wt_dtype;

/* Reading flags.  The default (WT_DEFAULT_FLAGS) is the reading under which
 * the method converges to the exact sorted composite as J grows. */
enum {
    /* Visibility at a fragment excludes the fragment's own step: v is the
     * transmittance in front of the interface (§1.2: v = 1 up to the plane,
     * 0.75 beyond it). */
    WT_SELF_EXCLUDE = 1u,
    /* Reconstruct A(z) by linear interpolation between the bin centres
     * (m + 1/2)/C, constant outside [c_0, c_{C-1}] (§2.3.2); off = staircase. */
    WT_INTERP_LINEAR = 2u,
    /* Normalised weighted resolve rgb = (R/W)(1 - T) + bg T; off = the literal
     * compositing sum of §2.2, rgb = sum c_i alpha_i v(z_i) + bg T. */
    WT_RESOLVE_NORMALIZED = 4u,
    /* wt_build / wt_resolve add into coeff / accum instead of overwriting
     * (several draw batches of one frame). */
    WT_ACCUMULATE = 8u
};
#define WT_DEFAULT_FLAGS (WT_SELF_EXCLUDE | WT_INTERP_LINEAR | WT_RESOLVE_NORMALIZED)

/* Frame descriptor. */
typedef struct wt_desc {
    int32_t width, height;  /* image size in pixels, each >= 1, width*height < 2^31 */
    int32_t tile_w, tile_h; /* screen tile that groups the fragment stream;
                               1 <= tile_w * tile_h <= 256; tiles are row-major,
                               ntiles = ceil(width/tile_w) * ceil(height/tile_h) */
    int32_t J;              /* Haar levels, 1..6; C = 2^J coefficients per pixel.
                               The coloured call (wt_build_resolve_rgb) and the
                               allocation-free batch stop at J = 5.
                               The paper's rank N is J - 1 (Wavelet3: J = 4) */
    int32_t coeff_dtype;    /* wt_dtype */
    uint32_t flags;         /* WT_* reading flags */
    int32_t reserved;       /* must be 0 */
} wt_desc;

/* Fragment stream, structure of arrays, device memory.  Fragments are grouped
 * by tile: tile t owns [tile_offsets[t], tile_offsets[t+1]).  The order inside
 * a tile is arbitrary (the method is order independent). */
typedef struct wt_frags {
    int64_t n;                   /* number of fragments, >= 0 */
    const uint32_t *pixel;       /* [n] pixel id y*width + x */
    const float *z;              /* [n] normalised depth */
    const float *alpha;          /* [n] opacity */
    const float *r, *g, *b;      /* [n] surface colour (not premultiplied);
                                    may be NULL for wt_build */
    const int64_t *tile_offsets; /* [ntiles + 1], non-decreasing, last = n */
} wt_frags;

/* Library version string (static storage). */
const char *wt_version(void);

/* Human-readable name of a status (static storage). */
const char *wt_status_string(wt_status s);

/* Bytes of the coefficient buffer: width*height * 2^J * sizeof(dtype), plus
 * width*height exponent bytes for WT_SE16 (sizeof = 2); 0 if the descriptor
 * is invalid. */
size_t wt_coeff_bytes(const wt_desc *desc);

/* Number of tiles of the descriptor (the length of tile_offsets minus one);
 * 0 if the descriptor is invalid. */
int64_t wt_num_tiles(const wt_desc *desc);

/*
 * wt_build -- §2.1 step 2 with §2.3.1 ("Coefficients").
 * For every pixel p computes, in FP32, the closed-form Haar projection of
 * A_p(z) = sum_i a_i theta(z - z_i) (§2.2):
 *     chi_00 = sum a_i (1 - z_i),   X_{n,k} = -sum a_i Psi_{n,k}(z_i),
 * with Psi_{n,k} the tent antiderivative of psi_{n,k}, and stores it once in
 * coeff_dtype (round to nearest even).
 *   coeff [P * C] of coeff_dtype, written (or added to under WT_ACCUMULATE);
 *         pixels without fragments get zeros.
 *   zmin  [P] float, nullable.  The nearest clamped depth of a fragment with
 *         alpha > 0 (+inf if none), i.e. the near half of the tight per-pixel
 *         depth bounds of §2.1 step 1; under WT_ACCUMULATE the minimum with
 *         the stored value.  wt_resolve uses it to keep the normalised
 *         resolve free of FP32 underflow in very deep pixels.
 *   total [P] float, nullable.  The pixel's total step S = sum a_i (0 if it
 *         has no fragments), from the same fixed-point bins as the
 *         coefficients (the sum of the root's two bins, exact up to one FP32
 *         rounding); under WT_ACCUMULATE added to the stored value.  Given to
 *         wt_resolve / wt_resolve_composite, it spares them summing the steps
 *         again fragment by fragment.
 * frags->r, g, b are not read.
 */
wt_status wt_build(const wt_desc *desc, const wt_frags *frags, void *coeff, float *zmin,
                   float *total, wt_stream stream);

/*
 * wt_resolve -- §2.1 step 3 with §2.2 and §2.3.2 ("Interpolation").
 * For every fragment: A_i = reconstruction of the pixel's coefficients at z_i
 * (minus the fragment's own step under WT_SELF_EXCLUDE), v_i = exp(-A_i),
 * w_i = alpha_i v_i; per pixel accumulates R,G,B = sum c_i w_i, W = sum w_i
 * and S = sum a_i.
 *   coeff [P * C] as written by wt_build (same desc).
 *   zmin  [P] from wt_build, nullable.  Under WT_RESOLVE_NORMALIZED and with
 *         zmin given, R, G, B and W of a pixel are all multiplied by the same
 *         positive factor exp(m_p) (m_p fixed by coeff and zmin), so only the
 *         ratios R/W, G/W, B/W are meaningful; without zmin m_p = 0.  In the
 *         literal mode m_p = 0 always.
 *   total [P] from wt_build, nullable.  If given, S is taken from it instead
 *         of being summed over the fragments (the own step removed under
 *         WT_SELF_EXCLUDE is then -log2(1 - alpha) from the hardware log2, as
 *         in wt_build_resolve).  Not accepted under WT_ACCUMULATE
 *         (WT_ERR_UNSUPPORTED): total covers every batch of the frame.
 *   accum [P * 5] float {R, G, B, W, S} per pixel, written (or added to under
 *         WT_ACCUMULATE: batches of one frame share m_p).
 */
wt_status wt_resolve(const wt_desc *desc, const wt_frags *frags, const void *coeff,
                     const float *zmin, const float *total, float *accum, wt_stream stream);

/*
 * wt_composite -- §2.1 step 4 (composite over the opaque background).
 * T = exp(-S).  WT_RESOLVE_NORMALIZED: rgb = (R/W)(1 - T) + bg T, or bg where
 * W = 0.  Literal: rgb = R + bg T.  In both: out.a = 1 - T.
 *   accum  [P * 5] from wt_resolve.
 *   bg_img [P * 3] float background image, nullable (then bg is used).
 *   bg     host pointer to 3 floats, used when bg_img is NULL.
 *   out    [P * 4] float RGBA.
 */
wt_status wt_composite(const wt_desc *desc, const float *accum, const float *bg_img,
                       const float bg[3], float *out, wt_stream stream);

/*
 * wt_composite_ca -- step 4 (§2.1) with the chromatic-aberration approximation
 * of §3.  The background term samples bg_img not once at the refracted point
 * p + d (d = offset[p], the pixel's screen-space refraction offset in pixels,
 * accumulated by the caller during shading) but at `taps` points along a
 * segment aligned with d and proportional to it:
 *   x_i = p + s_i d,  s_i = 1 + dispersion (t_i - 1/2),  t_i = i / (taps - 1),
 * bilinear samples (texel centres at integer + 1/2, clamped to the edge),
 * and each channel is the mean of the samples under its spectral weight,
 *   w_r = smoothstep(1/2, 1/3, t), w_b = smoothstep(1/2, 2/3, t),
 *   w_g = 1 - w_r - w_b
 * (§3's listing with the taps spread over t in [0, 1]; the smoothstep formula
 * is applied as written for the falling edge).  Then rgb and alpha as in
 * wt_composite with that background.
 *   accum      [P * 5] from wt_resolve.
 *   bg_img     [P * 3] float background image (required).
 *   offset     [P * 2] float (dx, dy), 8-byte aligned, nullable (no offset).
 *              A non-finite offset is replaced by 0 and counted in the error
 *              word.
 *   dispersion >= 0: the segment's length as a fraction of |d|.
 *   taps       1 (the single refracted sample) or odd, 3..15 (the paper: 5).
 *   out        [P * 4] float RGBA.
 * Only width, height and WT_RESOLVE_NORMALIZED of desc are used; images more
 * than 1048560 pixels high are WT_ERR_UNSUPPORTED.
 */
wt_status wt_composite_ca(const wt_desc *desc, const float *accum, const float *bg_img,
                          const float *offset, float dispersion, int32_t taps, float *out,
                          wt_stream stream);

/* wt_resolve followed by wt_composite in one kernel (no accum buffer); zmin
 * and total as for wt_resolve.  With both from wt_build (same desc), the
 * result equals wt_build_resolve's bit for bit. */
wt_status wt_resolve_composite(const wt_desc *desc, const wt_frags *frags, const void *coeff,
                               const float *zmin, const float *total, const float *bg_img,
                               const float bg[3], float *out, wt_stream stream);

/*
 * wt_build_resolve -- steps 2, 3 and 4 of §2.1 fused per screen tile: the
 * tile's coefficients are built in shared memory, rounded to coeff_dtype,
 * reconstructed and used for the resolve without a round trip through device
 * memory.  The result equals wt_build + wt_resolve_composite with the same
 * desc up to FP32 summation order.
 *   coeff [P * C] nullable: if given, the coefficients are also stored.
 *   zmin  [P] nullable: if given, the depth bound is also stored.
 *   out   [P * 4] float RGBA.
 *   accum [P * 5] float nullable: if given, the pixel sums {R, G, B, W, S}
 *         of the resolve are also stored (as wt_resolve's, with the weight
 *         offset m_p of the tile's near bound); wt_backward takes them to
 *         skip recomputing the forward sums.
 * WT_ACCUMULATE is not supported here (WT_ERR_UNSUPPORTED).
 */
wt_status wt_build_resolve(const wt_desc *desc, const wt_frags *frags, void *coeff, float *zmin,
                           const float *bg_img, const float bg[3], float *out, float *accum,
                           wt_stream stream);

/*
 * wt_build_resolve_tiles -- wt_build_resolve for the tiles
 * [first_tile, first_tile + num_tiles) only (tiles are independent, §2.1: the
 * method keeps constant state per pixel).  Only those tiles' fragment ranges
 * are read and only their pixels of coeff, zmin, out and accum are written, so a
 * caller can stream a frame in pieces, for example overlapping the upload of
 * the next range of tiles with the work on this one.  frags->tile_offsets
 * must still cover every tile.  A range outside [0, ntiles] is WT_ERR_ARG;
 * num_tiles = 0 launches nothing.
 */
wt_status wt_build_resolve_tiles(const wt_desc *desc, const wt_frags *frags, int64_t first_tile,
                                 int64_t num_tiles, void *coeff, float *zmin, const float *bg_img,
                                 const float bg[3], float *out, float *accum, wt_stream stream);

/*
 * wt_build_resolve_single_pass -- the single-pass variant the paper proposes
 * as future work (§4): frame t's fragments are resolved against frame t-1's
 * coefficients, which are complete before the call starts, and frame t's
 * coefficients are built for the next frame; nothing waits for this frame's
 * build.  Per screen tile the resolve comes first and the build second, each
 * fragment read from device memory once (the second read of a tile's range
 * is served by L2).  With an unchanged scene the composite equals
 * wt_build_resolve's; under motion the visibility is the previous frame's
 * (the paper's approximation; nothing is reprojected).
 *   coeff_prev [P * C] frame t-1's coefficients in coeff_dtype (the coeff
 *              output of the previous call, of wt_build or wt_build_resolve).
 *   zmin_prev  [P] nullable: frame t-1's near bound (the weight offset of
 *              the resolve comes from it; NULL = no offset).
 *   coeff      [P * C] nullable, written: frame t's coefficients; must not
 *              overlap coeff_prev (WT_ERR_ARG).
 *   zmin       [P] nullable, written: frame t's near bound.
 *   out        [P * 4] frame t's composite.
 * Weight exponents are clamped to [0, 120] (log2 units), so a fragment
 * nearer than anything in frame t-1, or hidden behind more than 120 log2
 * units of frame t-1's absorbance, keeps a finite, non-zero weight.
 * WT_ACCUMULATE is not supported here (WT_ERR_UNSUPPORTED).
 */
wt_status wt_build_resolve_single_pass(const wt_desc *desc, const wt_frags *frags, const void *coeff_prev,
                                       const float *zmin_prev, void *coeff, float *zmin,
                                       const float *bg_img, const float bg[3], float *out,
                                       wt_stream stream);

/* Storage of the coloured coefficients. */
enum {
    WT_RGB_F32 = 0,       /* float [3][P][C]: one plane per channel (r, g, b), each
                             laid out as the mono coefficient array */
    WT_RGB_E5B9G9R9 = 1   /* uint32 [P][C]: the three channels' magnitudes of each
                             coefficient index in one word: r in bits 0-8, g in
                             9-17, b in 18-26, a shared exponent e in 27-31,
                             value = mantissa * 2^(e - 24) (bias 15, no hidden
                             bit); chi_00 is stored as is, the X_{n,k} (all <= 0,
                             §2.3.1) as -X; 64 bytes per pixel at J = 4 */
};

/*
 * wt_build_resolve_rgb -- coloured absorbance: the three-channel form of the
 * method (§1.2, §2.1: the paper's coefficients carry r, g, b, packed
 * E5B9G9R9).  Fragment i has one depth z[i] and one opacity per channel,
 * alpha_r/g/b[i]; each channel is built and resolved as the mono method with
 * its own opacity and its own colour component,
 *   out_c = (R_c / W_c)(1 - T_c) + bg_c T_c  (WT_RESOLVE_NORMALIZED), with
 *   R_c = sum col_c alpha_c v_c(z), W_c = sum alpha_c v_c(z), T_c = exp(-sum a_c),
 * and out[p*4 + 3] = 1 - (T_r + T_g + T_b)/3.  Fused per tile like
 * wt_build_resolve; the resolve uses the coefficients rounded to coeff_format.
 *   frags        pixel, z, r, g, b and tile_offsets as usual (frags->alpha is
 *                not read).
 *   alpha_r/g/b  [n] per-channel opacity.
 *   coeff        nullable: written in coeff_format (WT_RGB_*).
 * With FP32 storage the channels are three launches of a one-channel fused
 * kernel (out's components are written one by one, out.w summed in channel
 * order); with E5B9G9R9 one CTA per tile works through the channels,
 * keeping r and g until the words are formed: as 16-bit magnitudes in the
 * pixel's own row of coeff (with its nearest depths and total steps in its out
 * entry) when coeff is given, as two FP32 rows per pixel in shared memory when
 * it is NULL.  Both give the same words and the same out bit for bit.  Every
 * tile of up to 256 pixels fits.
 * Invalid fragments (pixel outside their tile, NaN depth or a NaN opacity) are
 * left out of the channels they are invalid for and counted in the error word
 * once per channel.  WT_ACCUMULATE is not supported (WT_ERR_UNSUPPORTED).
 */
wt_status wt_build_resolve_rgb(const wt_desc *desc, const wt_frags *frags, const float *alpha_r,
                               const float *alpha_g, const float *alpha_b, void *coeff,
                               int32_t coeff_format, const float *bg_img, const float bg[3],
                               float *out, wt_stream stream);

/*
 * wt_build_resolve_batch_static -- wt_build_resolve for a batch of frames in
 * one launch, allocating nothing.  The paper has no counterpart: it exists for
 * callers that cannot allocate device memory when they submit work, such as a
 * renderer that reserves its whole device budget at start-up, or a real-time
 * loop in which cudaMalloc / cudaFree (which may synchronise the device) would
 * stall other work.  The scratch the launch needs -- per-frame parameters,
 * tile ranges and a work counter -- lives in a statically sized device array
 * of the library (about 13 KB, held by every GPU that loads the library until
 * the process exits); inputs and outputs are the caller's, and no
 * coefficients or depth bounds are stored.
 *   descs, frags  host arrays of nframes entries, 1 <= nframes <= 64 (larger
 *                 batches return WT_ERR_ARG).  All frames share J,
 *                 coeff_dtype and tile size (else WT_ERR_UNSUPPORTED);
 *                 WT_ACCUMULATE is not accepted.
 *   bgs           host array of nframes * 3 background colours.
 *   outs          host array of nframes device pointers, out[k] of [P_k * 4].
 * The first call on a device resolves the scratch's device address with that
 * device current (cudaGetSymbolAddress); make that first call before any
 * stream capture begins.  Every call reuses
 * the same scratch (each call re-initialises all of it that it uses, the
 * counter included): calls that overlap on the GPU -- on different streams,
 * or from different host threads without ordering -- race on it.
 */
wt_status wt_build_resolve_batch_static(const wt_desc *descs, const wt_frags *frags,
                                        const float *bgs, float *const *outs, int32_t nframes,
                                        wt_stream stream);

/*
 * wt_absorbance -- the evaluation half of §2.3 ("... a logarithmic number of
 * coefficients ... Same applies during evaluation"): A(z) of pixel[q] at depth
 * z[q] for q queries, reading J+1 coefficients per bin.  With alpha non-NULL
 * and WT_SELF_EXCLUDE set, query q is treated as a fragment of that pixel and
 * its own step alpha[q] is removed, exactly as in wt_resolve.
 *   pixel [q], z [q], alpha [q] (nullable) device arrays; A_out [q] float.
 *   Queries with a bad pixel id or NaN depth return NaN and are counted.
 */
wt_status wt_absorbance(const wt_desc *desc, const void *coeff, int64_t q, const uint32_t *pixel,
                        const float *z, const float *alpha, float *A_out, wt_stream stream);

/*
 * wt_backward -- adjoint of wt_build_resolve (the paper has no gradient; this
 * follows from the linearity of the coefficients in the steps, §2.3.1).
 * Given dL/d(out) it returns dL/d(alpha) and dL/d(r, g, b) for every
 * fragment, treating depth as fixed.  Coefficients are rebuilt inside the
 * call from the fragments (nothing from the forward pass is stored), with the
 * same desc (J, storage rounding, flags) and background as the forward call.
 *   grad_out   [P * 4] float, dL/d(out RGBA).
 *   accum      [P * 5] float, nullable: the forward call's pixel sums, as
 *              stored by wt_build_resolve's accum with this desc, these
 *              fragments and this background; if given, the forward sums are
 *              not recomputed (one pass over the fragments fewer) and the
 *              result is the same.  Not checked against the fragments.
 *   grad_alpha [n] float, written; 0 where alpha is clamped (<= 0 or
 *              >= 1 - 2^-20) and for rejected fragments.  It holds
 *              intermediate values during the call, so it must not overlap
 *              any input or grad_rgb (WT_ERR_ARG).
 *   grad_rgb   [3 * n] float, planar: dL/dr at [0, n), dL/dg at [n, 2n),
 *              dL/db at [2n, 3n).
 * The pixel-level sums use FP32; WT_ACCUMULATE is not supported.
 */
wt_status wt_backward(const wt_desc *desc, const wt_frags *frags, const float *bg_img,
                      const float bg[3], const float *grad_out, const float *accum, float *grad_alpha,
                      float *grad_rgb, wt_stream stream);

/* ------------------------------------------------------------------------
 * Before the build: grouping an unordered stream by tile, and the per-pixel
 * depth bounds of §2.1 step 1 ("tight per-pixel depth bounds" of the
 * transparent surfaces, into which depth is normalised before the build).
 */

/* Bytes of device workspace wt_bin needs for n fragments with this
 * descriptor: a digit-count matrix (257 x ceil(n / 8192) counters) and, when
 * the tile ids need two 8-bit sort passes or more (more than 256 tiles), an
 * intermediate stream of 24 bytes and one digit byte per fragment (twice that
 * for more than 65536 tiles); 0 if the descriptor is invalid or n < 0.  Only
 * the descriptor's width, height, tile_w and tile_h are used. */
size_t wt_bin_workspace_bytes(const wt_desc *desc, int64_t n);

/*
 * wt_bin -- groups an unordered fragment stream by tile (row-major tiles of
 * desc) into caller-allocated output arrays: a stable radix sort by tile id,
 * 8 bits per pass (one pass for up to 256 tiles, two up to 65536, at most
 * four), each pass writing coalesced runs of fragments of one digit.
 *   in          n fragments in any order, n < 2^32 (else WT_ERR_ARG);
 *               in->tile_offsets is ignored (may be NULL); in->r/g/b may all
 *               be NULL (then r/g/b_out are unused).
 *   *_out       [n] device arrays (at least in->n elements each), written with
 *               the kept fragments grouped by tile; they must not overlap in.
 *   tile_offsets_out [ntiles + 1] int64, written: tile t owns
 *               [tile_offsets_out[t], tile_offsets_out[t+1]); the last entry
 *               is the number of kept fragments.
 *   workspace   device memory of workspace_bytes >= wt_bin_workspace_bytes(desc,
 *               in->n) bytes (else WT_ERR_ARG), 256-byte aligned, owned by the
 *               caller (overwritten).
 * Fragments whose pixel id is >= width*height are dropped and counted in the
 * error word.  The sort is stable: inside a tile the fragments keep their
 * input order, so the output is the same on every run.
 */
wt_status wt_bin(const wt_desc *desc, const wt_frags *in, uint32_t *pixel_out, float *z_out,
                 float *alpha_out, float *r_out, float *g_out, float *b_out,
                 int64_t *tile_offsets_out, void *workspace, size_t workspace_bytes,
                 wt_stream stream);

/*
 * wt_depth_bounds -- §2.1 step 1: per-pixel depth bounds of the transparent
 * fragments of a tile-grouped stream.
 *   zlo, zhi  [width*height] float, written: the smallest and largest raw depth
 *             of the pixel's fragments (NaN z or alpha and misfiled fragments
 *             excluded and counted); +inf / -inf for a pixel without any.
 * Only the descriptor's geometry is used.
 */
wt_status wt_depth_bounds(const wt_desc *desc, const wt_frags *frags, float *zlo, float *zhi,
                          wt_stream stream);

/*
 * wt_normalize_depth -- maps every fragment's raw depth into its pixel's
 * bounds: z_out = (z - zlo[p]) / (zhi[p] - zlo[p]) (FP32, IEEE division), and
 * 0 when the pixel's range is 0 or not finite.  The nearest fragment goes to 0
 * and the farthest to 1 (which the build clamps into the last bin).  Fragments
 * with a pixel id >= width*height or a NaN depth get NaN (the build then
 * rejects and counts them).  z_out may be frags->z (in place); the tile
 * grouping is not needed.
 */
wt_status wt_normalize_depth(const wt_desc *desc, const wt_frags *frags, const float *zlo,
                             const float *zhi, float *z_out, wt_stream stream);

/* ------------------------------------------------------------------------
 * Below the paper's passes: rasterising transparent particles (the smoke and
 * fire billboards of the paper's scenes, §3 and Fig. 2-3) into the fragment
 * stream that the calls above consume.
 */

/* Particles, structure of arrays, device memory.  Particle i is a
 * screen-space disc of centre (cx, cy) in pixel units (pixel (x, y) covers
 * [x, x+1) x [y, y+1)), radius `radius` pixels, normalised depth z, peak
 * opacity alpha and colour (r, g, b; all three may be NULL). */
typedef struct wt_particles {
    int64_t n;
    const float *cx, *cy, *radius, *z, *alpha;
    const float *r, *g, *b;
} wt_particles;

/* Bytes of device workspace of wt_raster_count / wt_raster_emit for n
 * particles (or triangles): n + 1 int64 offsets, then ceil(n / 4096) int64
 * partial sums of the count pass's scan. */
size_t wt_raster_workspace_bytes(int64_t n_particles);

/*
 * wt_raster_count -- first pass of the particle rasteriser.  A particle puts a
 * fragment on every pixel of the image whose centre (x + 1/2, y + 1/2) is at
 * squared distance d2 < radius^2 from (cx, cy), with opacity
 * alpha * (1 - d2 / radius^2) (every operation rounded separately in FP32, the
 * reciprocal of radius^2 taken once).  Writes into workspace (8-byte aligned,
 * wt_raster_workspace_bytes(n) bytes) the exclusive offsets of each particle's
 * fragments and, at [n], the total: read it back to size the fragment arrays
 * of wt_raster_emit; the bytes behind [n] are the scan's scratch.  Particles with
 * a non-positive or NaN radius, or a NaN centre, give no fragments.
 */
wt_status wt_raster_count(const wt_desc *desc, const wt_particles *particles, void *workspace,
                          wt_stream stream);

/*
 * wt_raster_emit -- second pass: writes the fragments, each particle's
 * contiguous at its offset, in particle order and row-major inside a particle
 * (the order a rasteriser submitting one particle after another produces),
 * into caller-allocated [capacity] arrays: pixel id y*width + x, the
 * particle's z and colour, the opacity above.  Fragments beyond capacity are
 * not written and are counted in the error word.  The stream is not grouped
 * by tile: wt_bin groups it.  Only the descriptor's width and height are used.
 */
wt_status wt_raster_emit(const wt_desc *desc, const wt_particles *particles, const void *workspace,
                         int64_t capacity, uint32_t *pixel, float *z, float *alpha, float *r,
                         float *g, float *b, wt_stream stream);

/* Screen-space triangles (glass panes: two per quad), device arrays.  Vertex
 * k of triangle i is (x, y, z)[3i + k] in pixel units and normalised depth;
 * opacity and colour are per triangle ([n]); r, g, b nullable together. */
typedef struct wt_triangles {
    int64_t n;
    const float *x, *y, *z;
    const float *alpha;
    const float *r, *g, *b;
} wt_triangles;

/*
 * wt_raster_tri_count -- first pass of the triangle rasteriser, the
 * counterpart of wt_raster_count (workspace of wt_raster_workspace_bytes(n)).
 * Coverage is exact: vertices are snapped to 1/256 pixel (X = rint(256 x),
 * ties to even) and the pixel centre C = (256 x + 128, 256 y + 128) is inside
 * when every integer edge function E(A->B) = (Bx-Ax)(Cy-Ay) - (By-Ay)(Cx-Ax)
 * of the triangle, wound to positive area, is > 0, or = 0 on an edge with
 * dy < 0, or dy = 0 and dx > 0 (a centre on an edge or vertex shared by
 * triangles that tile the plane belongs to exactly one of them).  Zero-area
 * triangles, non-finite vertices and |x| or |y| >= 2^22 give no fragments.
 * Images of width or height >= 2^21 are WT_ERR_UNSUPPORTED.
 */
wt_status wt_raster_tri_count(const wt_desc *desc, const wt_triangles *triangles, void *workspace,
                              wt_stream stream);

/*
 * wt_raster_tri_emit -- second pass, as wt_raster_emit: fragments in triangle
 * order, row-major inside a triangle, with the triangle's opacity and colour
 * and the depth z = ((e0 z0 + e1 z1) + e2 z2) / area, where e_k is the edge
 * function opposite vertex k and area the doubled area, each converted to
 * FP32 and every operation rounded separately in FP32.
 */
wt_status wt_raster_tri_emit(const wt_desc *desc, const wt_triangles *triangles, const void *workspace,
                             int64_t capacity, uint32_t *pixel, float *z, float *alpha, float *r,
                             float *g, float *b, wt_stream stream);

/*
 * wt_get_error -- synchronises `stream`, then returns in *bad_count the
 * number of fragments (or queries, or tile ranges) rejected by any call on the
 * current device since the previous wt_get_error, and clears the count.
 * Returns WT_ERR_INPUT if the count was non-zero, WT_OK otherwise.
 */
wt_status wt_get_error(wt_stream stream, int64_t *bad_count);
/* (Every call counts the fragments it rejects, so a bad fragment seen by
 * wt_build and then by wt_resolve is counted twice.) */

/* ------------------------------------------------------------------------
 * Serving: continuous batching of frames on one GPU (no counterpart in the
 * paper, which renders one frame at a time).
 *
 * A server owns a device arena of mem_cap_bytes for the coefficient buffers
 * (allocated once by wt_serve_create; nothing is allocated per request) and a
 * scheduler thread.  Requests are admitted in arrival order while fewer than
 * max_slots are held and the held bytes -- fragments (24 B each) and tile
 * offsets, coefficients and output, counted per request -- stay under
 * mem_cap_bytes.  Each scheduling step is one persistent kernel launch over the
 * tiles of all admitted frames (an equal share of step_tiles each), so frames
 * that arrive while others are running are processed in the same launches.
 * The per-tile arithmetic is that of wt_build_resolve.  Kernels never wait on
 * the host; every host wait is bounded.
 */
typedef struct wt_serve_config {
    int32_t J, coeff_dtype; /* every request must use these ... */
    uint32_t flags;         /* ... and these reading flags ... */
    int32_t tile_w, tile_h; /* ... and this tile size */
    int32_t max_slots;      /* requests held at once (admitted, not released), 1..4096 */
    int64_t mem_cap_bytes;  /* byte cap for held requests; also the arena size */
    int64_t step_tiles;     /* tiles per scheduling step (one kernel launch) */
} wt_serve_config;

typedef struct wt_server wt_server;

typedef struct wt_serve_info {
    int32_t state;    /* 0 queued, 1 admitted, 2 done */
    int32_t reserved;
    double submit_us; /* host clock, microseconds since the server was created */
    double admit_us;  /* -1 if not admitted yet */
    double done_us;   /* GPU completion (from a CUDA event), -1 if not done */
    void *coeff;      /* the request's coefficient buffer in the arena (valid
                         until wt_serve_release), or NULL while queued */
} wt_serve_info;

/* Creates a server on the current device.  WT_ERR_CUDA if the arena or the
 * stream cannot be created. */
wt_status wt_serve_create(const wt_serve_config *cfg, wt_server **server);

/* Queues a frame.  desc must match the server's J, coeff_dtype, flags and tile
 * size (else WT_ERR_UNSUPPORTED).  The fragment arrays and out [P * 4] are the
 * caller's device memory and must stay valid until the request is done.
 * ready_stream is the stream on which they were produced: the server's work
 * for the request is ordered after everything enqueued there before this
 * call.  After wt_serve_wait returns WT_OK, out is complete for every stream.
 * WT_ERR_NOMEM if the frame alone exceeds the cap.  Thread safe. */
wt_status wt_serve_submit(wt_server *server, const wt_desc *desc, const wt_frags *frags,
                          const float bg[3], float *out, wt_stream ready_stream,
                          int64_t *request_id);

/* Waits until the request is done, at most timeout_us; WT_ERR_TIMEOUT if not. */
wt_status wt_serve_wait(wt_server *server, int64_t request_id, int64_t timeout_us);

/* State and timestamps of a request (see wt_serve_info). */
wt_status wt_serve_query(wt_server *server, int64_t request_id, wt_serve_info *info);

/* Gives back a done request's slot, bytes and coefficient buffer.
 * WT_ERR_ARG if the request is unknown or not done. */
wt_status wt_serve_release(wt_server *server, int64_t request_id);

/* Held bytes, queued and admitted-unfinished request counts; returns the
 * server's fault status (WT_OK normally). */
wt_status wt_serve_stats(wt_server *server, int64_t *used_bytes, int64_t *queued, int64_t *active);

/* Stops the scheduler, waits for the launched work and frees everything. */
wt_status wt_serve_destroy(wt_server *server);

/* The admission and step-planning policy of the server on its own, with no
 * GPU: for tests and for callers that drive their own launches.
 * wt_planner_submit returns a request id > 0 or -WT_ERR_NOMEM;
 * wt_planner_admit writes the newly admitted ids; wt_planner_plan writes one
 * step's tile ranges (id, first tile, count) and the ids whose last tiles are
 * in it (*nfinishing: capacity in, count out); both return their total
 * count. */
typedef struct wt_planner wt_planner;
wt_planner *wt_planner_create(int32_t max_slots, int64_t mem_cap_bytes, int64_t step_tiles);
int64_t wt_planner_submit(wt_planner *planner, int64_t bytes, int64_t tiles);
int32_t wt_planner_admit(wt_planner *planner, int64_t *ids, int32_t max_ids);
int32_t wt_planner_plan(wt_planner *planner, int64_t *ids, int32_t *tile0, int32_t *count,
                        int32_t max_ranges, int64_t *finishing, int32_t *nfinishing);
int32_t wt_planner_release(wt_planner *planner, int64_t request_id);
int64_t wt_planner_used(const wt_planner *planner);
void wt_planner_destroy(wt_planner *planner);

#ifdef __cplusplus
}
#endif
#endif /* WT_H */
