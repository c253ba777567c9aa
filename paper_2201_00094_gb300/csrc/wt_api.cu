// C-ABI entry points of libwt.so (declared in include/wt.h): argument
// validation on the host, dispatch to the per-J / per-dtype kernels, and the
// per-device error word that counts rejected fragments.
#include <mutex>

#include "wt.h"
#include "wt_internal.h"
#include "wt_trace.h"
#include "wt_tile.cuh"

namespace wt {

// Count of rejected fragments / queries / tile ranges.  One per device (every
// device that loads the library holds this 8-byte word).
__device__ unsigned long long g_bad_count;

namespace {

constexpr int kMaxDevices = 64;
unsigned long long *g_err_ptr[kMaxDevices];
std::once_flag g_err_once[kMaxDevices];

// Device address of g_bad_count on the current device (resolved once per device).
unsigned long long *err_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::call_once(g_err_once[dev], [dev] {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_bad_count) == cudaSuccess)
            g_err_ptr[dev] = static_cast<unsigned long long *>(ptr);
    });
    return g_err_ptr[dev];
}

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

bool dtype_ok(int32_t dt) { return dt == WT_F32 || dt == WT_BF16 || dt == WT_F16 || dt == WT_SE16; }

// Validates the descriptor; returns WT_OK or the reason.
wt_status check_desc(const wt_desc *d) {
    if (!d) return WT_ERR_ARG;
    if (d->width < 1 || d->height < 1) return WT_ERR_ARG;
    if ((int64_t)d->width * d->height >= (int64_t(1) << 31)) return WT_ERR_ARG;
    if (d->tile_w < 1 || d->tile_h < 1 || (int64_t)d->tile_w * d->tile_h > kMaxTilePx) return WT_ERR_ARG;
    if (d->J < 1) return WT_ERR_ARG;
    if (d->J > kMaxJ) return WT_ERR_UNSUPPORTED;
    if (!dtype_ok(d->coeff_dtype)) return WT_ERR_ARG;
    if (d->flags & ~uint32_t(WT_SELF_EXCLUDE | WT_INTERP_LINEAR | WT_RESOLVE_NORMALIZED | WT_ACCUMULATE))
        return WT_ERR_ARG;
    if (d->reserved != 0) return WT_ERR_ARG;
    return WT_OK;
}

int64_t ntiles_of(const wt_desc *d) {
    const int64_t ntx = (d->width + d->tile_w - 1) / d->tile_w;
    const int64_t nty = (d->height + d->tile_h - 1) / d->tile_h;
    return ntx * nty;
}

wt_status check_frags(const wt_frags *f, bool need_rgb) {
    if (!f || f->n < 0 || !f->tile_offsets) return WT_ERR_ARG;
    if (!aligned(f->tile_offsets, 8)) return WT_ERR_ARG;
    const void *req[3] = {f->pixel, f->z, f->alpha};
    for (const void *p : req)
        if ((f->n > 0 && !p) || !aligned(p, 16)) return WT_ERR_ARG;
    if (need_rgb) {
        const void *col[3] = {f->r, f->g, f->b};
        for (const void *p : col)
            if ((f->n > 0 && !p) || !aligned(p, 16)) return WT_ERR_ARG;
    }
    return WT_OK;
}

Params make_params(const wt_desc *d, const wt_frags *f) {
    Params p{};
    p.g.width = d->width;
    p.g.height = d->height;
    p.g.tile_w = d->tile_w;
    p.g.tile_h = d->tile_h;
    p.g.ntx = (d->width + d->tile_w - 1) / d->tile_w;
    p.flags = d->flags;
    set_row_division(p);
    if (f) {
        p.n = f->n;
        p.pixel = f->pixel;
        p.z = f->z;
        p.alpha = f->alpha;
        p.r = f->r;
        p.gc = f->g;
        p.b = f->b;
        p.off = f->tile_offsets;
    }
    p.bg0 = p.bg1 = p.bg2 = 0.f;
    return p;
}

const TileLaunch *table(const TileLaunch *t0, const TileLaunch *t1, const TileLaunch *t2, const TileLaunch *t3,
                        int dt) {
    return by_dtype(dt, t0, t1, t2, t3);
}

// A launcher returns cudaErrorNotSupported for a layout beyond the shared
// memory of one CTA (a large J with a large tile), before anything is launched.
wt_status finish(cudaError_t e) {
    return e == cudaSuccess ? WT_OK : (e == cudaErrorNotSupported ? WT_ERR_UNSUPPORTED : WT_ERR_CUDA);
}

wt_status set_bg(Params &p, const float *bg_img, const float *bg) {
    if (bg_img) {
        if (!aligned(bg_img, 4)) return WT_ERR_ARG;
        p.bg_img = bg_img;
    } else {
        if (!bg) return WT_ERR_ARG;
        p.bg0 = bg[0];
        p.bg1 = bg[1];
        p.bg2 = bg[2];
    }
    return WT_OK;
}

// Step 4 from an accumulation buffer: one thread per pixel.
__global__ void __launch_bounds__(kThreads) k_composite(Params p) {
    const int64_t P = (int64_t)p.g.width * p.g.height;
    for (int64_t gp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gp < P;
         gp += (int64_t)gridDim.x * blockDim.x) {
        const float *a = p.accum + 5 * gp;
        composite_pixel(p, gp, a[0], a[1], a[2], a[3], a[4]);
    }
}

}  // namespace

// Device address of the error word on the current device (for other units).
unsigned long long *error_word() { return err_word(); }

}  // namespace wt

using namespace wt;

extern "C" {

const char *wt_version(void) { return "wt-gb300 0.1 (sm_103a)"; }

const char *wt_status_string(wt_status s) {
    switch (s) {
    case WT_OK: return "ok";
    case WT_ERR_ARG: return "invalid argument";
    case WT_ERR_UNSUPPORTED: return "unsupported";
    case WT_ERR_INPUT: return "rejected input fragments";
    case WT_ERR_TIMEOUT: return "timeout";
    case WT_ERR_CUDA: return "CUDA error";
    case WT_ERR_NOMEM: return "over memory cap";
    case WT_ERR_BUSY: return "busy";
    default: return "unknown status";
    }
}

size_t wt_coeff_bytes(const wt_desc *d) {
    if (check_desc(d) != WT_OK) return 0;
    return coeff_storage_bytes((int64_t)d->width * d->height, d->J, d->coeff_dtype);
}

int64_t wt_num_tiles(const wt_desc *d) { return check_desc(d) == WT_OK ? ntiles_of(d) : 0; }

wt_status wt_build(const wt_desc *d, const wt_frags *f, void *coeff, float *zmin, float *total,
                   wt_stream stream) {
    WT_TRACE();
    wt_status st = check_desc(d);
    if (st != WT_OK) return st;
    if ((st = check_frags(f, false)) != WT_OK) return st;
    if (!coeff || !aligned(coeff, 16) || (zmin && !aligned(zmin, 4)) || (total && !aligned(total, 4)))
        return WT_ERR_ARG;
    Params p = make_params(d, f);
    p.coeff = coeff;
    p.zmin = zmin;
    p.total = total;
    if (!(p.err = err_word())) return WT_ERR_CUDA;
    const TileLaunch *t = table(kBuild0, kBuild1, kBuild2, kBuild3, d->coeff_dtype);
    return finish(t[d->J - 1](p, (int)ntiles_of(d), reinterpret_cast<cudaStream_t>(stream)));
}

wt_status wt_resolve(const wt_desc *d, const wt_frags *f, const void *coeff, const float *zmin,
                     const float *total, float *accum, wt_stream stream) {
    WT_TRACE();
    wt_status st = check_desc(d);
    if (st != WT_OK) return st;
    if ((st = check_frags(f, true)) != WT_OK) return st;
    if (!coeff || !aligned(coeff, 16) || !accum || !aligned(accum, 4) || (zmin && !aligned(zmin, 4)) ||
        (total && !aligned(total, 4)))
        return WT_ERR_ARG;
    if (total && (d->flags & WT_ACCUMULATE)) return WT_ERR_UNSUPPORTED;  // total covers every batch
    Params p = make_params(d, f);
    p.coeff = const_cast<void *>(coeff);
    p.zmin = const_cast<float *>(zmin);
    p.total = const_cast<float *>(total);
    p.accum = accum;
    if (!(p.err = err_word())) return WT_ERR_CUDA;
    const TileLaunch *t = table(kResolve0, kResolve1, kResolve2, kResolve3, d->coeff_dtype);
    return finish(t[d->J - 1](p, (int)ntiles_of(d), reinterpret_cast<cudaStream_t>(stream)));
}

wt_status wt_composite(const wt_desc *d, const float *accum, const float *bg_img, const float bg[3],
                       float *out, wt_stream stream) {
    WT_TRACE();
    wt_status st = check_desc(d);
    if (st != WT_OK) return st;
    if (!accum || !aligned(accum, 4) || !out || !aligned(out, 16)) return WT_ERR_ARG;
    Params p = make_params(d, nullptr);
    p.accum = const_cast<float *>(accum);
    p.out = out;
    if ((st = set_bg(p, bg_img, bg)) != WT_OK) return st;
    const int64_t P = (int64_t)d->width * d->height;
    const int blocks = (int)((P + kThreads - 1) / kThreads < 152 * 8 ? (P + kThreads - 1) / kThreads : 152 * 8);
    k_composite<<<blocks, kThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(p);
    return finish(cudaGetLastError());
}

wt_status wt_resolve_composite(const wt_desc *d, const wt_frags *f, const void *coeff,
                               const float *zmin, const float *total, const float *bg_img, const float bg[3],
                               float *out, wt_stream stream) {
    WT_TRACE();
    wt_status st = check_desc(d);
    if (st != WT_OK) return st;
    if ((st = check_frags(f, true)) != WT_OK) return st;
    if (!coeff || !aligned(coeff, 16) || !out || !aligned(out, 16) || (zmin && !aligned(zmin, 4)) ||
        (total && !aligned(total, 4)))
        return WT_ERR_ARG;
    if (total && (d->flags & WT_ACCUMULATE)) return WT_ERR_UNSUPPORTED;
    Params p = make_params(d, f);
    p.coeff = const_cast<void *>(coeff);
    p.zmin = const_cast<float *>(zmin);
    p.total = const_cast<float *>(total);
    p.out = out;
    if ((st = set_bg(p, bg_img, bg)) != WT_OK) return st;
    if (!(p.err = err_word())) return WT_ERR_CUDA;
    const TileLaunch *t = table(kResolveComp0, kResolveComp1, kResolveComp2, kResolveComp3, d->coeff_dtype);
    return finish(t[d->J - 1](p, (int)ntiles_of(d), reinterpret_cast<cudaStream_t>(stream)));
}

wt_status wt_build_resolve_tiles(const wt_desc *d, const wt_frags *f, int64_t first_tile, int64_t num_tiles,
                                 void *coeff, float *zmin, const float *bg_img, const float bg[3], float *out,
                                 float *accum, wt_stream stream) {
    WT_TRACE();
    wt_status st = check_desc(d);
    if (st != WT_OK) return st;
    if (d->flags & WT_ACCUMULATE) return WT_ERR_UNSUPPORTED;
    if ((st = check_frags(f, true)) != WT_OK) return st;
    if ((coeff && !aligned(coeff, 16)) || !out || !aligned(out, 16) || (zmin && !aligned(zmin, 4)) ||
        (accum && !aligned(accum, 4)))
        return WT_ERR_ARG;
    const int64_t nt = ntiles_of(d);
    if (first_tile < 0 || num_tiles < 0 || first_tile + num_tiles > nt) return WT_ERR_ARG;
    if (num_tiles == 0) return WT_OK;
    Params p = make_params(d, f);
    p.tile0 = (int32_t)first_tile;
    p.coeff = coeff;
    p.zmin = zmin;
    p.out = out;
    p.accum = accum;
    if ((st = set_bg(p, bg_img, bg)) != WT_OK) return st;
    if (!(p.err = err_word())) return WT_ERR_CUDA;
    const TileLaunch *t = table(kFused0, kFused1, kFused2, kFused3, d->coeff_dtype);
    return finish(t[d->J - 1](p, (int)num_tiles, reinterpret_cast<cudaStream_t>(stream)));
}

wt_status wt_build_resolve_single_pass(const wt_desc *d, const wt_frags *f, const void *coeff_prev,
                                       const float *zmin_prev, void *coeff, float *zmin, const float *bg_img,
                                       const float bg[3], float *out, wt_stream stream) {
    WT_TRACE();
    wt_status st = check_desc(d);
    if (st != WT_OK) return st;
    if (d->flags & WT_ACCUMULATE) return WT_ERR_UNSUPPORTED;
    if ((st = check_frags(f, true)) != WT_OK) return st;
    if (!coeff_prev || !aligned(coeff_prev, 16) || (coeff && !aligned(coeff, 16)) || !out || !aligned(out, 16) ||
        (zmin && !aligned(zmin, 4)) || (zmin_prev && !aligned(zmin_prev, 4)))
        return WT_ERR_ARG;
    // frame t's outputs must not overlap frame t-1's inputs
    const size_t cb = coeff_storage_bytes((int64_t)d->width * d->height, d->J, d->coeff_dtype);
    const char *cp = static_cast<const char *>(coeff_prev), *cn = static_cast<const char *>(coeff);
    if (coeff && cn < cp + cb && cp < cn + cb) return WT_ERR_ARG;
    if (zmin && zmin_prev && zmin == zmin_prev) return WT_ERR_ARG;
    Params p = make_params(d, f);
    p.coeff = coeff;
    p.zmin = zmin;
    p.out = out;
    if ((st = set_bg(p, bg_img, bg)) != WT_OK) return st;
    if (!(p.err = err_word())) return WT_ERR_CUDA;
    const TemporalLaunch *t = by_dtype(d->coeff_dtype, kTemporal0, kTemporal1, kTemporal2, kTemporal3);
    return finish(t[d->J - 1](p, (int)ntiles_of(d), coeff_prev, zmin_prev, reinterpret_cast<cudaStream_t>(stream)));
}

wt_status wt_build_resolve_rgb(const wt_desc *d, const wt_frags *f, const float *alpha_r, const float *alpha_g,
                               const float *alpha_b, void *coeff, int32_t coeff_format, const float *bg_img,
                               const float bg[3], float *out, wt_stream stream) {
    WT_TRACE();
    wt_status st = check_desc(d);
    if (st != WT_OK) return st;
    if (d->flags & WT_ACCUMULATE) return WT_ERR_UNSUPPORTED;
    if (coeff_format != WT_RGB_F32 && coeff_format != WT_RGB_E5B9G9R9) return WT_ERR_ARG;
    if (d->J > 5) return WT_ERR_UNSUPPORTED;  // the coloured kernels stop at 32 coefficients
    if (!f || f->n < 0 || !f->tile_offsets || !aligned(f->tile_offsets, 8)) return WT_ERR_ARG;
    const void *req[8] = {f->pixel, f->z, f->r, f->g, f->b, alpha_r, alpha_g, alpha_b};
    for (const void *q : req)  // 16-byte aligned: the fragment passes read them as vectors
        if ((f->n > 0 && !q) || !aligned(q, 16)) return WT_ERR_ARG;
    if ((coeff && !aligned(coeff, 16)) || !out || !aligned(out, 16)) return WT_ERR_ARG;
    const int npx = d->tile_w * d->tile_h;
    if (rgb_smem_bytes(d->J, npx, coeff_format == WT_RGB_E5B9G9R9) > 227 * 1024) return WT_ERR_UNSUPPORTED;
    Params p = make_params(d, f);
    p.coeff = coeff;
    p.out = out;
    if ((st = set_bg(p, bg_img, bg)) != WT_OK) return st;
    if (!(p.err = err_word())) return WT_ERR_CUDA;
    const float *const ac[3] = {alpha_r, alpha_g, alpha_b};
    return finish(launch_fused_rgb(p, d->J, ac, coeff_format == WT_RGB_E5B9G9R9, (int)ntiles_of(d),
                                   reinterpret_cast<cudaStream_t>(stream)));
}

wt_status wt_build_resolve(const wt_desc *d, const wt_frags *f, void *coeff, float *zmin,
                           const float *bg_img, const float bg[3], float *out, float *accum, wt_stream stream) {
    WT_TRACE();
    wt_status st = check_desc(d);
    if (st != WT_OK) return st;
    return wt_build_resolve_tiles(d, f, 0, ntiles_of(d), coeff, zmin, bg_img, bg, out, accum, stream);
}

wt_status wt_backward(const wt_desc *d, const wt_frags *f, const float *bg_img, const float bg[3],
                      const float *grad_out, const float *accum, float *grad_alpha, float *grad_rgb,
                      wt_stream stream) {
    WT_TRACE();
    wt_status st = check_desc(d);
    if (st != WT_OK) return st;
    if (d->flags & WT_ACCUMULATE) return WT_ERR_UNSUPPORTED;
    if ((st = check_frags(f, true)) != WT_OK) return st;
    if (!grad_out || !aligned(grad_out, 16)) return WT_ERR_ARG;
    if (f->n > 0 && (!grad_alpha || !grad_rgb)) return WT_ERR_ARG;
    if (!aligned(grad_alpha, 4) || !aligned(grad_rgb, 4) || (accum && !aligned(accum, 4))) return WT_ERR_ARG;
    // grad_alpha holds intermediate values while the fragments are still
    // being read, so it must not overlap any input
    {
        const size_t nb = (size_t)f->n * 4, pb = (size_t)d->width * d->height;
        const char *ga = reinterpret_cast<const char *>(grad_alpha);
        auto overlaps = [&](const void *q, size_t qb) {
            const char *c = static_cast<const char *>(q);
            return c && nb && qb && ga < c + qb && c < ga + nb;
        };
        if (overlaps(f->pixel, nb) || overlaps(f->z, nb) || overlaps(f->alpha, nb) || overlaps(f->r, nb) ||
            overlaps(f->g, nb) || overlaps(f->b, nb) || overlaps(f->tile_offsets, (size_t)(ntiles_of(d) + 1) * 8) ||
            overlaps(grad_out, pb * 16) || overlaps(bg_img, pb * 12) || overlaps(accum, pb * 20) ||
            overlaps(grad_rgb, 3 * nb))
            return WT_ERR_ARG;
    }
    Params p = make_params(d, f);
    if ((st = set_bg(p, bg_img, bg)) != WT_OK) return st;
    p.gout = grad_out;
    p.accum = const_cast<float *>(accum);
    p.galpha = grad_alpha;
    p.grgb = grad_rgb;
    if (!(p.err = err_word())) return WT_ERR_CUDA;
    const TileLaunch *t = table(kBackward0, kBackward1, kBackward2, kBackward3, d->coeff_dtype);
    return finish(t[d->J - 1](p, (int)ntiles_of(d), reinterpret_cast<cudaStream_t>(stream)));
}

wt_status wt_absorbance(const wt_desc *d, const void *coeff, int64_t q, const uint32_t *pixel,
                        const float *z, const float *alpha, float *A_out, wt_stream stream) {
    WT_TRACE();
    wt_status st = check_desc(d);
    if (st != WT_OK) return st;
    if (q < 0 || !coeff || !aligned(coeff, 4)) return WT_ERR_ARG;
    if (q > 0 && (!pixel || !z || !A_out)) return WT_ERR_ARG;
    Params p = make_params(d, nullptr);
    p.coeff = const_cast<void *>(coeff);
    if (!(p.err = err_word())) return WT_ERR_CUDA;
    const QueryLaunch *t = by_dtype(d->coeff_dtype, kAbsorbance0, kAbsorbance1, kAbsorbance2, kAbsorbance3);
    return finish(t[d->J - 1](p, q, pixel, z, alpha, A_out, reinterpret_cast<cudaStream_t>(stream)));
}

wt_status wt_get_error(wt_stream stream, int64_t *bad_count) {
    WT_TRACE();
    if (!bad_count) return WT_ERR_ARG;
    unsigned long long *w = err_word();
    if (!w) return WT_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned long long host = 0;
    if (cudaMemcpyAsync(&host, w, sizeof(host), cudaMemcpyDeviceToHost, s) != cudaSuccess) return WT_ERR_CUDA;
    if (cudaMemsetAsync(w, 0, sizeof(host), s) != cudaSuccess) return WT_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return WT_ERR_CUDA;
    *bad_count = (int64_t)host;
    return host ? WT_ERR_INPUT : WT_OK;
}

}  // extern "C"
