// The layer below the paper's passes: rasterising transparent primitives into
// the fragment stream that the build and resolve consume.  Two primitives:
//
// * Particles (smoke billboards): a screen-space disc, centre (cx, cy) in
//   pixel units, radius rho, one depth z, a peak opacity alpha0 and a colour.
//   It puts a fragment on every pixel whose centre (x + 1/2, y + 1/2) lies
//   strictly inside the disc, with the opacity falling off to zero at the rim:
//       d2 = dx*dx + dy*dy,  covered iff d2 < rho*rho,
//       alpha = alpha0 * (1 - d2 * (1 / (rho*rho))),
//   every operation rounded separately in FP32 (no contraction), so that the
//   same decisions and values come out of any FP32 implementation.
//
// * Triangles (glass panes, two per quad), with per-vertex depth and a flat
//   opacity and colour.  Coverage is exact: the vertices are snapped to 1/256
//   pixel and the edge functions of the pixel centre are integers.  A centre
//   on an edge belongs to the triangle it enters when moved right and
//   infinitesimally down, so triangles that share edges or vertices cover
//   every centre once.  Depth comes from the barycentric weights in a fixed
//   sequence of FP32 operations.
//
// One warp per primitive walks the primitive's clipped bounding box in
// row-major order, 32 pixels at a time: a counting pass, a scan of the
// counts, and an emitting pass that writes each primitive's fragments
// contiguously, in that order.
#include "wt.h"
#include "wt_internal.h"
#include "wt_trace.h"
#include "wt_tile.cuh"

namespace wt {

unsigned long long *error_word();  // wt_api.cu

namespace {

struct RasterGeom {
    int width, height;
};

struct RasterOut {
    uint32_t *pixel;
    float *z, *alpha, *r, *g, *b;
    int64_t capacity;
};

// ---------------------------------------------------------------- particles

struct Particles {
    int64_t n;
    const float *cx, *cy, *radius, *z, *alpha, *r, *g, *b;
};

// A particle's clipped bounding box and its disc parameters.
struct Disc {
    int x0, y0, w, h;  // box origin and extent (w or h 0: nothing)
    float cx, cy, rho2, inv, z, a0;

    // Whether pixel (x, y) is covered, and the fragment's depth and opacity.
    __device__ __forceinline__ bool cover(int x, int y, float &zf, float &af) const {
        const float dx = __fsub_rn(__fadd_rn((float)x, 0.5f), cx);
        const float dy = __fsub_rn(__fadd_rn((float)y, 0.5f), cy);
        const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        zf = z;
        af = __fmul_rn(a0, __fsub_rn(1.f, __fmul_rn(d2, inv)));
        return d2 < rho2;
    }
};

struct DiscPrim {
    using Input = Particles;
    using Shape = Disc;
    static __device__ __forceinline__ Disc make(const Particles &pt, int64_t i, const RasterGeom &g) {
        Disc d{};
        const float cx = pt.cx[i], cy = pt.cy[i], rho = pt.radius[i];
        if (!(rho > 0.f) || !(cx == cx) || !(cy == cy) || !(rho < 1e6f) || !(fabsf(cx) < 1e9f) ||
            !(fabsf(cy) < 1e9f))
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
        d.z = pt.z[i];
        d.a0 = pt.alpha[i];
        return d;
    }
};

// ---------------------------------------------------------------- triangles

struct Triangles {
    int64_t n;
    const float *x, *y, *z, *alpha, *r, *g, *b;
};

// A triangle snapped to 1/256 pixel and wound so that its doubled area is
// positive, with its clipped bounding box.
struct Tri {
    int x0, y0, w, h;
    long long X[3], Y[3];
    float z[3], area, a0;

    // Edge k is the edge opposite vertex k: (1, 2), (2, 0), (0, 1).  Its
    // function at the centre is the weight of vertex k times the doubled area.
    __device__ __forceinline__ bool cover(int x, int y, float &zf, float &af) const {
        const long long cx = 256ll * x + 128, cy = 256ll * y + 128;
        long long E[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int a = k == 2 ? 0 : k + 1, b = k == 0 ? 2 : (k == 1 ? 0 : 1);
            const long long dx = X[b] - X[a], dy = Y[b] - Y[a];
            E[k] = dx * (cy - Y[a]) - dy * (cx - X[a]);
        }
        bool in = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int a = k == 2 ? 0 : k + 1, b = k == 0 ? 2 : (k == 1 ? 0 : 1);
            const long long dx = X[b] - X[a], dy = Y[b] - Y[a];
            in &= E[k] > 0 || (E[k] == 0 && (dy < 0 || (dy == 0 && dx > 0)));
        }
        const float e0 = __ll2float_rn(E[0]), e1 = __ll2float_rn(E[1]), e2 = __ll2float_rn(E[2]);
        zf = __fdiv_rn(__fadd_rn(__fadd_rn(__fmul_rn(e0, z[0]), __fmul_rn(e1, z[1])), __fmul_rn(e2, z[2])), area);
        af = a0;
        return in;
    }
};

struct TriPrim {
    using Input = Triangles;
    using Shape = Tri;
    static __device__ __forceinline__ Tri make(const Triangles &t, int64_t i, const RasterGeom &g) {
        Tri s{};
        float vx[3], vy[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            vx[k] = t.x[3 * i + k];
            vy[k] = t.y[3 * i + k];
            s.z[k] = t.z[3 * i + k];
            if (!(fabsf(vx[k]) < 4194304.f) || !(fabsf(vy[k]) < 4194304.f)) return s;  // also NaN
            // x * 256 is exact; rounding to the nearest integer, ties to even
            s.X[k] = __float2ll_rn(vx[k] * 256.f);
            s.Y[k] = __float2ll_rn(vy[k] * 256.f);
        }
        long long area = (s.X[1] - s.X[0]) * (s.Y[2] - s.Y[0]) - (s.Y[1] - s.Y[0]) * (s.X[2] - s.X[0]);
        if (area == 0) return s;
        if (area < 0) {
            long long tx = s.X[1], ty = s.Y[1];
            s.X[1] = s.X[2];
            s.Y[1] = s.Y[2];
            s.X[2] = tx;
            s.Y[2] = ty;
            const float tz = s.z[1];
            s.z[1] = s.z[2];
            s.z[2] = tz;
            area = -area;
        }
        const long long mnx = min(s.X[0], min(s.X[1], s.X[2])), mxx = max(s.X[0], max(s.X[1], s.X[2]));
        const long long mny = min(s.Y[0], min(s.Y[1], s.Y[2])), mxy = max(s.Y[0], max(s.Y[1], s.Y[2]));
        // candidate centres 256 p + 128 in [min, max]: floor((min - 128) / 256) .. floor((max - 128) / 256) + 1
        const long long x0 = max(0ll, (mnx - 128) >> 8), x1 = min((long long)g.width - 1, ((mxx - 128) >> 8) + 1);
        const long long y0 = max(0ll, (mny - 128) >> 8), y1 = min((long long)g.height - 1, ((mxy - 128) >> 8) + 1);
        if (x1 < x0 || y1 < y0) return s;
        s.x0 = (int)x0;
        s.y0 = (int)y0;
        s.w = (int)(x1 - x0 + 1);
        s.h = (int)(y1 - y0 + 1);
        s.area = __ll2float_rn(area);
        s.a0 = t.alpha[i];
        return s;
    }
};

// ---------------------------------------------------------------- the walk

template <class Prim>
__global__ void __launch_bounds__(256) k_raster_count(RasterGeom g, typename Prim::Input in, int64_t *__restrict__ counts) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < in.n; i += nw) {
        const typename Prim::Shape s = Prim::make(in, i, g);
        const int64_t area = (int64_t)s.w * s.h;
        int64_t c = 0;
        for (int64_t q0 = 0; q0 < area; q0 += 32) {
            const int64_t q = q0 + lane;
            bool hit = false;
            if (q < area) {
                float zf, af;
                hit = s.cover(s.x0 + (int)(q % s.w), s.y0 + (int)(q / s.w), zf, af);
            }
            c += __popc(__ballot_sync(0xffffffffu, hit));
        }
        if (lane == 0) counts[i] = c;
    }
}

// Exclusive scan of n counts in place into offsets[0 .. n] (offsets[n] = the
// total), in three launches: each block scans a chunk of kScanChunk counts
// and leaves the chunk's total in part[]; one block scans the totals; every
// chunk adds its offset.
constexpr int kScanThreads = 1024, kScanItems = 4, kScanChunk = kScanThreads * kScanItems;

// Block-wide exclusive scan of one value per thread; *total gets the sum.
__device__ __forceinline__ long long block_exclusive_scan(long long v, long long *total) {
    __shared__ long long warp_sum[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sum[w] = x;
    __syncthreads();
    if (w == 0) {
        long long t = lane < kScanThreads / 32 ? warp_sum[lane] : 0ll;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < kScanThreads / 32) warp_sum[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const long long before = w > 0 ? warp_sum[w - 1] : 0ll;
    *total = warp_sum[kScanThreads / 32 - 1];
    __syncthreads();  // warp_sum is reused by the next call
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_chunks(int64_t n, int64_t *__restrict__ v,
                                                              long long *__restrict__ part) {
    const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
    long long x[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        x[k] = base + k < n ? v[base + k] : 0ll;
        s += x[k];
    }
    long long total;
    long long run = block_exclusive_scan(s, &total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) v[base + k] = run;
        run += x[k];
    }
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// One block: exclusive scan of the nb chunk totals in place, rounds of
// kScanThreads; v[n] = the grand total.
__global__ void __launch_bounds__(kScanThreads) k_scan_parts(int64_t nb, long long *__restrict__ part, int64_t n,
                                                             int64_t *__restrict__ v) {
    long long carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        const int64_t i = b0 + threadIdx.x;
        const long long x = i < nb ? part[i] : 0ll;
        long long total;
        const long long e = block_exclusive_scan(x, &total);
        if (i < nb) part[i] = carry + e;
        carry += total;
    }
    if (threadIdx.x == 0) v[n] = carry;
}

__global__ void __launch_bounds__(256) k_scan_add(int64_t n, int64_t *__restrict__ v,
                                                  const long long *__restrict__ part) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] += part[i / kScanChunk];
}

// The scan's chunk totals behind the n + 1 offsets.
__host__ __device__ constexpr int64_t scan_parts(int64_t n) { return (n + kScanChunk - 1) / kScanChunk; }

void scan_offsets(int64_t n, int64_t *offsets, cudaStream_t s) {
    long long *part = reinterpret_cast<long long *>(offsets + n + 1);
    const int64_t nb = scan_parts(n);
    if (nb > 0) k_scan_chunks<<<(unsigned)nb, kScanThreads, 0, s>>>(n, offsets, part);
    k_scan_parts<<<1, kScanThreads, 0, s>>>(nb, part, n, offsets);
    if (nb > 1) k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, offsets, part);
}

template <class Prim>
__global__ void __launch_bounds__(256) k_raster_emit(RasterGeom g, typename Prim::Input in,
                                                     const int64_t *__restrict__ offsets, RasterOut o,
                                                     unsigned long long *err) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long dropped = 0;
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < in.n; i += nw) {
        const typename Prim::Shape s = Prim::make(in, i, g);
        const int64_t area = (int64_t)s.w * s.h;
        const float cr = in.r ? in.r[i] : 0.f, cg = in.g ? in.g[i] : 0.f, cb = in.b ? in.b[i] : 0.f;
        int64_t at = offsets[i];
        for (int64_t q0 = 0; q0 < area; q0 += 32) {
            const int64_t q = q0 + lane;
            bool hit = false;
            float zf = 0.f, af = 0.f;
            int x = 0, y = 0;
            if (q < area) {
                x = s.x0 + (int)(q % s.w);
                y = s.y0 + (int)(q / s.w);
                hit = s.cover(x, y, zf, af);
            }
            const unsigned m = __ballot_sync(0xffffffffu, hit);
            const int64_t slot = at + __popc(m & lt);
            if (hit) {
                if (slot < o.capacity) {
                    o.pixel[slot] = (uint32_t)y * (uint32_t)g.width + (uint32_t)x;
                    o.z[slot] = zf;
                    o.alpha[slot] = af;
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

wt_status check_geom(const wt_desc *desc) {
    if (!desc || desc->width < 1 || desc->height < 1) return WT_ERR_ARG;
    if ((int64_t)desc->width * desc->height >= (int64_t(1) << 31)) return WT_ERR_ARG;
    return WT_OK;
}

wt_status check_particles(const wt_desc *desc, const wt_particles *p) {
    if (check_geom(desc) != WT_OK) return WT_ERR_ARG;
    if (!p || p->n < 0) return WT_ERR_ARG;
    if (p->n > 0 && (!p->cx || !p->cy || !p->radius || !p->z || !p->alpha)) return WT_ERR_ARG;
    const bool rgb = p->r != nullptr;
    if (rgb != (p->g != nullptr) || rgb != (p->b != nullptr)) return WT_ERR_ARG;
    return WT_OK;
}

wt_status check_triangles(const wt_desc *desc, const wt_triangles *t) {
    if (check_geom(desc) != WT_OK) return WT_ERR_ARG;
    // pixel centres in 1/256 units stay below 2^30, so every edge function fits 64 bits
    if (desc->width >= (1 << 21) || desc->height >= (1 << 21)) return WT_ERR_UNSUPPORTED;
    if (!t || t->n < 0) return WT_ERR_ARG;
    if (t->n > 0 && (!t->x || !t->y || !t->z || !t->alpha)) return WT_ERR_ARG;
    const bool rgb = t->r != nullptr;
    if (rgb != (t->g != nullptr) || rgb != (t->b != nullptr)) return WT_ERR_ARG;
    return WT_OK;
}

Particles particles_of(const wt_particles *p) {
    return Particles{p->n, p->cx, p->cy, p->radius, p->z, p->alpha, p->r, p->g, p->b};
}

Triangles triangles_of(const wt_triangles *t) { return Triangles{t->n, t->x, t->y, t->z, t->alpha, t->r, t->g, t->b}; }

template <class Prim>
wt_status count_t(const wt_desc *desc, const typename Prim::Input &in, void *workspace, wt_stream stream) {
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 7)) return WT_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t *offsets = static_cast<int64_t *>(workspace);
    const RasterGeom g{desc->width, desc->height};
    if (in.n > 0) k_raster_count<Prim><<<warps_grid(in.n), 256, 0, s>>>(g, in, offsets);
    scan_offsets(in.n, offsets, s);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

template <class Prim>
wt_status emit_t(const wt_desc *desc, const typename Prim::Input &in, const void *workspace, int64_t capacity,
                 uint32_t *pixel, float *z, float *alpha, float *r, float *g, float *b, wt_stream stream) {
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 7) || capacity < 0) return WT_ERR_ARG;
    if (capacity > 0 && (!pixel || !z || !alpha)) return WT_ERR_ARG;
    const bool rgb = in.r != nullptr;
    if (rgb && capacity > 0 && (!r || !g || !b)) return WT_ERR_ARG;
    unsigned long long *err = error_word();
    if (!err) return WT_ERR_CUDA;
    if (in.n == 0) return WT_OK;
    const RasterGeom geo{desc->width, desc->height};
    const RasterOut o{pixel, z, alpha, rgb ? r : nullptr, rgb ? g : nullptr, rgb ? b : nullptr, capacity};
    k_raster_emit<Prim><<<warps_grid(in.n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        geo, in, static_cast<const int64_t *>(workspace), o, err);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

}  // namespace
}  // namespace wt

using namespace wt;

extern "C" size_t wt_raster_workspace_bytes(int64_t n_particles) {
    return n_particles < 0 ? 0 : (size_t)(n_particles + 1 + scan_parts(n_particles)) * 8;
}

extern "C" wt_status wt_raster_count(const wt_desc *desc, const wt_particles *particles, void *workspace,
                                     wt_stream stream) {
    WT_TRACE();
    wt_status st = check_particles(desc, particles);
    if (st != WT_OK) return st;
    return count_t<DiscPrim>(desc, particles_of(particles), workspace, stream);
}

extern "C" wt_status wt_raster_emit(const wt_desc *desc, const wt_particles *particles, const void *workspace,
                                    int64_t capacity, uint32_t *pixel, float *z, float *alpha, float *r, float *g,
                                    float *b, wt_stream stream) {
    WT_TRACE();
    wt_status st = check_particles(desc, particles);
    if (st != WT_OK) return st;
    return emit_t<DiscPrim>(desc, particles_of(particles), workspace, capacity, pixel, z, alpha, r, g, b, stream);
}

extern "C" wt_status wt_raster_tri_count(const wt_desc *desc, const wt_triangles *triangles, void *workspace,
                                         wt_stream stream) {
    WT_TRACE();
    wt_status st = check_triangles(desc, triangles);
    if (st != WT_OK) return st;
    return count_t<TriPrim>(desc, triangles_of(triangles), workspace, stream);
}

extern "C" wt_status wt_raster_tri_emit(const wt_desc *desc, const wt_triangles *triangles, const void *workspace,
                                        int64_t capacity, uint32_t *pixel, float *z, float *alpha, float *r,
                                        float *g, float *b, wt_stream stream) {
    WT_TRACE();
    wt_status st = check_triangles(desc, triangles);
    if (st != WT_OK) return st;
    return emit_t<TriPrim>(desc, triangles_of(triangles), workspace, capacity, pixel, z, alpha, r, g, b, stream);
}
