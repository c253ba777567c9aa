// The layer below the paper's passes: rasterising transparent particle
// billboards into the fragment stream that the build and resolve consume.
//
// A particle is a screen-space disc: centre (cx, cy) in pixel units, radius
// rho, one depth z, a peak opacity alpha0 and a colour.  It puts a fragment on
// every pixel whose centre (x + 1/2, y + 1/2) lies strictly inside the disc,
// with the opacity falling off to zero at the rim:
//     d2 = dx*dx + dy*dy,  covered iff d2 < rho*rho,
//     alpha = alpha0 * (1 - d2 * (1 / (rho*rho))),
// every operation rounded separately in FP32 (no contraction), so that the
// same decisions and values come out of any FP32 implementation.
//
// One warp per particle walks the particle's clipped bounding box in
// row-major order, 32 pixels at a time: a counting pass, a scan of the
// counts, and an emitting pass that writes each particle's fragments
// contiguously, in that order.
#include "wt.h"
#include "wt_internal.h"
#include "wt_tile.cuh"

namespace wt {

unsigned long long *error_word();  // wt_api.cu

namespace {

struct RasterGeom {
    int width, height;
};

struct Particles {
    int64_t n;
    const float *cx, *cy, *radius, *z, *alpha, *r, *g, *b;
};

// A particle's clipped bounding box and its disc parameters.
struct Disc {
    int x0, y0, w, h;  // box origin and extent (w or h 0: nothing)
    float cx, cy, rho2, inv;
};

__device__ __forceinline__ Disc disc_of(const Particles &pt, int64_t i, const RasterGeom &g) {
    Disc d{};
    const float cx = pt.cx[i], cy = pt.cy[i], rho = pt.radius[i];
    if (!(rho > 0.f) || !(cx == cx) || !(cy == cy) || !(rho < 1e6f) || !(fabsf(cx) < 1e9f) || !(fabsf(cy) < 1e9f))
        return d;  // no area, or coordinates outside any sensible screen
    // pixel centres inside the disc satisfy |x + 1/2 - cx| < rho; the box is
    // widened by a pixel on each side so that rounding here never drops one
    // (the distance test alone decides coverage)
    const int x0 = max(0, (int)floorf(cx - rho - 0.5f) - 1), x1 = min(g.width - 1, (int)ceilf(cx + rho - 0.5f) + 1);
    const int y0 = max(0, (int)floorf(cy - rho - 0.5f) - 1), y1 = min(g.height - 1, (int)ceilf(cy + rho - 0.5f) + 1);
    if (x1 < x0 || y1 < y0) return d;
    d.x0 = x0;
    d.y0 = y0;
    d.w = x1 - x0 + 1;
    d.h = y1 - y0 + 1;
    d.cx = cx;
    d.cy = cy;
    d.rho2 = __fmul_rn(rho, rho);
    d.inv = __fdiv_rn(1.f, d.rho2);
    return d;
}

// Squared distance of pixel (x, y)'s centre to the disc centre.
__device__ __forceinline__ float dist2(const Disc &d, int x, int y) {
    const float dx = __fsub_rn(__fadd_rn((float)x, 0.5f), d.cx);
    const float dy = __fsub_rn(__fadd_rn((float)y, 0.5f), d.cy);
    return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
}

__global__ void __launch_bounds__(256) k_raster_count(RasterGeom g, Particles pt, int64_t *__restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < pt.n; i += nw) {
        const Disc d = disc_of(pt, i, g);
        const int64_t area = (int64_t)d.w * d.h;
        int64_t c = 0;
        for (int64_t q0 = 0; q0 < area; q0 += 32) {
            const int64_t q = q0 + lane;
            bool in = false;
            if (q < area) in = dist2(d, d.x0 + (int)(q % d.w), d.y0 + (int)(q / d.w)) < d.rho2;
            c += __popc(__ballot_sync(0xffffffffu, in));
        }
        if (lane == 0) counts[i] = c;
    }
}

// One block: exclusive scan of n counts in place into offsets[0 .. n], each
// thread scanning a contiguous chunk.
__global__ void __launch_bounds__(1024) k_raster_scan(int64_t n, int64_t *__restrict__ offsets) {
    __shared__ long long part[1024];
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t b = threadIdx.x * per, e = min(n, b + per);
    long long sum = 0;
    for (int64_t t = b; t < e; ++t) sum += offsets[t];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int dd = 1; dd < (int)blockDim.x; dd <<= 1) {
        const long long v = threadIdx.x >= (unsigned)dd ? part[threadIdx.x - dd] : 0ll;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    long long run = part[threadIdx.x] - sum;
    for (int64_t t = b; t < e; ++t) {
        const long long c = offsets[t];
        offsets[t] = run;
        run += c;
    }
    if (threadIdx.x == blockDim.x - 1) offsets[n] = part[threadIdx.x];
}

struct RasterOut {
    uint32_t *pixel;
    float *z, *alpha, *r, *g, *b;
    int64_t capacity;
};

__global__ void __launch_bounds__(256) k_raster_emit(RasterGeom g, Particles pt, const int64_t *__restrict__ offsets,
                                                     RasterOut o, unsigned long long *err) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long dropped = 0;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < pt.n; i += nw) {
        const Disc d = disc_of(pt, i, g);
        const int64_t area = (int64_t)d.w * d.h;
        const float z = pt.z[i], a0 = pt.alpha[i];
        const float cr = pt.r ? pt.r[i] : 0.f, cg = pt.g ? pt.g[i] : 0.f, cb = pt.b ? pt.b[i] : 0.f;
        int64_t at = offsets[i];
        for (int64_t q0 = 0; q0 < area; q0 += 32) {
            const int64_t q = q0 + lane;
            bool in = false;
            float d2 = 0.f;
            int x = 0, y = 0;
            if (q < area) {
                x = d.x0 + (int)(q % d.w);
                y = d.y0 + (int)(q / d.w);
                d2 = dist2(d, x, y);
                in = d2 < d.rho2;
            }
            const unsigned m = __ballot_sync(0xffffffffu, in);
            const int64_t slot = at + __popc(m & lt);
            if (in) {
                if (slot < o.capacity) {
                    o.pixel[slot] = (uint32_t)y * (uint32_t)g.width + (uint32_t)x;
                    o.z[slot] = z;
                    o.alpha[slot] = __fmul_rn(a0, __fsub_rn(1.f, __fmul_rn(d2, d.inv)));
                    if (o.r) {
                        o.r[slot] = cr;
                        o.g[slot] = cg;
                        o.b[slot] = cb;
                    }
                } else {
                    ++dropped;
                }
            }
            at += __popc(m);
        }
    }
    if (dropped) atomicAdd(err, dropped);
}

int warps_grid(int64_t n) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 7) / 8;  // 8 warps per block
    const int64_t cap = (int64_t)sms * 16;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

wt_status check_particles(const wt_desc *desc, const wt_particles *p) {
    if (!desc || desc->width < 1 || desc->height < 1) return WT_ERR_ARG;
    if ((int64_t)desc->width * desc->height >= (int64_t(1) << 31)) return WT_ERR_ARG;
    if (!p || p->n < 0) return WT_ERR_ARG;
    if (p->n > 0 && (!p->cx || !p->cy || !p->radius || !p->z || !p->alpha)) return WT_ERR_ARG;
    const bool rgb = p->r != nullptr;
    if (rgb != (p->g != nullptr) || rgb != (p->b != nullptr)) return WT_ERR_ARG;
    return WT_OK;
}

Particles particles_of(const wt_particles *p) {
    return Particles{p->n, p->cx, p->cy, p->radius, p->z, p->alpha, p->r, p->g, p->b};
}

}  // namespace
}  // namespace wt

using namespace wt;

extern "C" size_t wt_raster_workspace_bytes(int64_t n_particles) {
    return n_particles < 0 ? 0 : (size_t)(n_particles + 1) * 8;
}

extern "C" wt_status wt_raster_count(const wt_desc *desc, const wt_particles *particles, void *workspace,
                                     wt_stream stream) {
    wt_status st = check_particles(desc, particles);
    if (st != WT_OK) return st;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 7)) return WT_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t *offsets = static_cast<int64_t *>(workspace);
    const RasterGeom g{desc->width, desc->height};
    if (particles->n > 0)
        k_raster_count<<<warps_grid(particles->n), 256, 0, s>>>(g, particles_of(particles), offsets);
    k_raster_scan<<<1, 1024, 0, s>>>(particles->n, offsets);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

extern "C" wt_status wt_raster_emit(const wt_desc *desc, const wt_particles *particles, const void *workspace,
                                    int64_t capacity, uint32_t *pixel, float *z, float *alpha, float *r, float *g,
                                    float *b, wt_stream stream) {
    wt_status st = check_particles(desc, particles);
    if (st != WT_OK) return st;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 7) || capacity < 0) return WT_ERR_ARG;
    if (capacity > 0 && (!pixel || !z || !alpha)) return WT_ERR_ARG;
    const bool rgb = particles->r != nullptr;
    if (rgb && capacity > 0 && (!r || !g || !b)) return WT_ERR_ARG;
    unsigned long long *err = error_word();
    if (!err) return WT_ERR_CUDA;
    if (particles->n == 0) return WT_OK;
    const RasterGeom geo{desc->width, desc->height};
    const RasterOut o{pixel, z, alpha, rgb ? r : nullptr, rgb ? g : nullptr, rgb ? b : nullptr, capacity};
    k_raster_emit<<<warps_grid(particles->n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        geo, particles_of(particles), static_cast<const int64_t *>(workspace), o, err);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}
