// Step 4 (§2.1) with the chromatic-aberration approximation of §3: the
// background behind the transparent layers is not one bilinear sample at the
// refracted point p + d (d: the pixel's screen-space refraction offset,
// accumulated during shading) but `taps` bilinear samples along a segment
// aligned with d and proportional to it,
//     x_i = p + s_i d,  s_i = 1 + dispersion (t_i - 1/2),  t_i = i / (taps - 1),
// each colour channel taking the mean of the samples under its spectral
// weight: w_r = smoothstep(1/2, 1/3, t), w_b = smoothstep(1/2, 2/3, t),
// w_g = 1 - w_r - w_b (the smoothstep formula applied as written for the
// falling edge).  Red then comes from one end of the segment, blue from the
// other, green from the middle.  The composite over that background is step
// 4's.
//
// A block per 64 x 16 tile of pixels, with the background under the tile and
// a halo staged in shared memory (taps beyond the halo read global memory).
#include <math.h>

#include "wt.h"
#include "wt_internal.h"
#include "wt_trace.h"
#include "wt_tile.cuh"

namespace wt {

unsigned long long *error_word();  // wt_api.cu

namespace {

constexpr int kMaxTaps = 15;

struct CaParams {
    int width, height;
    uint32_t flags;
    const float *__restrict__ accum;   // [P][5] R, G, B, W, S
    const float *__restrict__ bg;      // [P][3]
    const float2 *__restrict__ offset; // [P] (dx, dy), nullable
    float *out;                        // [P][4]
    unsigned long long *err;
    float s[kMaxTaps];     // tap positions along d
    float w[kMaxTaps][3];  // spectral weights, each channel's column summing to 1
};

// The bilinear combination of four texels (t00 at (i0, j0), t10 at (i0 + 1, j0), ...).
__device__ __forceinline__ float3 blend(float ax, float ay, float3 t00, float3 t10, float3 t01, float3 t11) {
    const float w00 = (1.f - ax) * (1.f - ay), w10 = ax * (1.f - ay), w01 = (1.f - ax) * ay, w11 = ax * ay;
    float3 v;
    v.x = w00 * t00.x + w10 * t10.x + w01 * t01.x + w11 * t11.x;
    v.y = w00 * t00.y + w10 * t10.y + w01 * t01.y + w11 * t11.y;
    v.z = w00 * t00.z + w10 * t10.z + w01 * t01.z + w11 * t11.z;
    return v;
}

__device__ __forceinline__ float3 texel(const float *bg, int64_t k) {
    return make_float3(__ldg(bg + 3 * k), __ldg(bg + 3 * k + 1), __ldg(bg + 3 * k + 2));
}

// Bilinear sample of the RGB background from global memory at the texel
// corner (x0, y0) = floor of the position minus 1/2, weights (ax, ay), clamped
// to the edge; corners far outside the image are clamped before the integer
// conversion.
__device__ __forceinline__ float3 bilinear_global(const CaParams &q, float x0, float y0, float ax, float ay) {
    x0 = fminf(fmaxf(x0, -1.f), (float)q.width);
    y0 = fminf(fmaxf(y0, -1.f), (float)q.height);
    const int ia = (int)x0, ja = (int)y0;
    const int i0 = min(max(ia, 0), q.width - 1), i1 = min(max(ia + 1, 0), q.width - 1);
    const int64_t j0 = min(max(ja, 0), q.height - 1), j1 = min(max(ja + 1, 0), q.height - 1);
    return blend(ax, ay, texel(q.bg, j0 * q.width + i0), texel(q.bg, j0 * q.width + i1),
                 texel(q.bg, j1 * q.width + i0), texel(q.bg, j1 * q.width + i1));
}

// A block composites a 64 x 16 tile of pixels (256 threads, four rows each)
// and first stages the background under the tile and a 12-pixel halo in
// shared memory, one plane per channel, texels clamped to the image as the
// global path clamps them.  A tap whose four texels lie in the staged region
// reads them there (the same values the global path reads); others read
// global memory.
constexpr int kCaTW = 64, kCaTH = 16, kCaHalo = 12;
constexpr int kCaRW = kCaTW + 2 * kCaHalo + 1, kCaRH = kCaTH + 2 * kCaHalo + 1;

template <int TAPS> __global__ void __launch_bounds__(256) k_composite_ca(CaParams q) {
    __shared__ float sbg[3][kCaRH][kCaRW];
    const int tx0 = blockIdx.x * kCaTW, ty0 = blockIdx.y * kCaTH;
    const int rx0 = tx0 - kCaHalo, ry0 = ty0 - kCaHalo;
    for (int t = threadIdx.x; t < kCaRW * kCaRH; t += blockDim.x) {
        const int rj = t / kCaRW, ri = t - rj * kCaRW;
        const int gx = min(max(rx0 + ri, 0), q.width - 1), gy = min(max(ry0 + rj, 0), q.height - 1);
        const float3 v = texel(q.bg, (int64_t)gy * q.width + gx);
        sbg[0][rj][ri] = v.x;
        sbg[1][rj][ri] = v.y;
        sbg[2][rj][ri] = v.z;
    }
    __syncthreads();
    auto staged = [&](int ri, int rj) { return make_float3(sbg[0][rj][ri], sbg[1][rj][ri], sbg[2][rj][ri]); };
    unsigned bad = 0;
    const int lx = threadIdx.x % kCaTW;
#pragma unroll 1
    for (int ly = threadIdx.x / kCaTW; ly < kCaTH; ly += blockDim.x / kCaTW) {
        const int x = tx0 + lx, y = ty0 + ly;
        if (x >= q.width || y >= q.height) continue;
        const int64_t gp = (int64_t)y * q.width + x;
        float2 d = q.offset ? q.offset[gp] : make_float2(0.f, 0.f);
        if (!(fabsf(d.x) <= 3.4e38f) || !(fabsf(d.y) <= 3.4e38f)) {  // NaN or infinite: no shift
            d = make_float2(0.f, 0.f);
            ++bad;
        }
        const float cx = (float)x + 0.5f, cy = (float)y + 0.5f;
        float3 bgc = make_float3(0.f, 0.f, 0.f);
#pragma unroll
        for (int i = 0; i < TAPS; ++i) {
            const float fx = fmaf(q.s[i], d.x, cx) - 0.5f, fy = fmaf(q.s[i], d.y, cy) - 0.5f;
            const float x0 = floorf(fx), y0 = floorf(fy);
            const float ax = fx - x0, ay = fy - y0;
            const float rxf = x0 - (float)rx0, ryf = y0 - (float)ry0;
            float3 v;
            if (rxf >= 0.f && rxf <= (float)(kCaRW - 2) && ryf >= 0.f && ryf <= (float)(kCaRH - 2)) {
                const int ri = (int)rxf, rj = (int)ryf;
                v = blend(ax, ay, staged(ri, rj), staged(ri + 1, rj), staged(ri, rj + 1), staged(ri + 1, rj + 1));
            } else {
                v = bilinear_global(q, x0, y0, ax, ay);
            }
            bgc.x = fmaf(q.w[i][0], v.x, bgc.x);
            bgc.y = fmaf(q.w[i][1], v.y, bgc.y);
            bgc.z = fmaf(q.w[i][2], v.z, bgc.z);
        }
        const float *a = q.accum + 5 * gp;
        const float R = a[0], G = a[1], B = a[2], W = a[3], S = a[4];
        const float T = ex2(-S * kLog2e);
        const float cover = S < 0.0009765625f ? S * fmaf(-0.5f, S, 1.f) : 1.f - T;
        float4 o;
        if (q.flags & kNormalized) {
            if (W > 0.f) {
                const float k = W >= 1.17549435e-38f ? cover * rcp(W) : cover / W;
                o.x = fmaf(R, k, bgc.x * T);
                o.y = fmaf(G, k, bgc.y * T);
                o.z = fmaf(B, k, bgc.z * T);
            } else {
                o.x = bgc.x;
                o.y = bgc.y;
                o.z = bgc.z;
            }
        } else {
            o.x = fmaf(bgc.x, T, R);
            o.y = fmaf(bgc.y, T, G);
            o.z = fmaf(bgc.z, T, B);
        }
        o.w = cover;
        reinterpret_cast<float4 *>(q.out)[gp] = o;
    }
    flush_bad(bad, q.err);
}

template <int TAPS> cudaError_t launch_ca(const CaParams &q, cudaStream_t s) {
    const dim3 grid((q.width + kCaTW - 1) / kCaTW, (q.height + kCaTH - 1) / kCaTH);
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    k_composite_ca<TAPS><<<grid, 256, 0, s>>>(q);
    return cudaGetLastError();
}

// The GLSL smoothstep formula, also for a falling edge (e0 > e1).
double smoothstep(double e0, double e1, double x) {
    double u = (x - e0) / (e1 - e0);
    u = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
    return u * u * (3.0 - 2.0 * u);
}

}  // namespace
}  // namespace wt

using namespace wt;

extern "C" wt_status wt_composite_ca(const wt_desc *desc, const float *accum, const float *bg_img,
                                     const float *offset, float dispersion, int32_t taps, float *out,
                                     wt_stream stream) {
    WT_TRACE();
    if (!desc || desc->width < 1 || desc->height < 1 || desc->reserved != 0) return WT_ERR_ARG;
    if ((int64_t)desc->width * desc->height >= (int64_t(1) << 31)) return WT_ERR_ARG;
    if (!accum || (reinterpret_cast<uintptr_t>(accum) & 3) || !bg_img || (reinterpret_cast<uintptr_t>(bg_img) & 3))
        return WT_ERR_ARG;
    if ((offset && (reinterpret_cast<uintptr_t>(offset) & 7)) || !out || (reinterpret_cast<uintptr_t>(out) & 15))
        return WT_ERR_ARG;
    if (taps < 1 || taps > kMaxTaps || taps % 2 == 0) return WT_ERR_ARG;
    if (!(dispersion >= 0.f) || !(dispersion <= 3.4e38f)) return WT_ERR_ARG;
    if ((desc->height + kCaTH - 1) / kCaTH > 65535) return WT_ERR_UNSUPPORTED;  // rows of the launch grid
    CaParams q{};
    q.width = desc->width;
    q.height = desc->height;
    q.flags = desc->flags;
    q.accum = accum;
    q.bg = bg_img;
    q.offset = reinterpret_cast<const float2 *>(offset);
    q.out = out;
    if (!(q.err = error_word())) return WT_ERR_CUDA;
    // tap positions and weights (one tap: the plain refracted sample)
    double w[kMaxTaps][3], sum[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < taps; ++i) {
        const double t = taps == 1 ? 0.5 : (double)i / (taps - 1);
        q.s[i] = (float)(1.0 + (double)dispersion * (t - 0.5));
        if (taps == 1) {
            w[i][0] = w[i][1] = w[i][2] = 1.0;
        } else {
            w[i][0] = smoothstep(0.5, 1.0 / 3.0, t);
            w[i][2] = smoothstep(0.5, 2.0 / 3.0, t);
            w[i][1] = 1.0 - w[i][0] - w[i][2];
        }
        for (int c = 0; c < 3; ++c) sum[c] += w[i][c];
    }
    for (int i = 0; i < taps; ++i)
        for (int c = 0; c < 3; ++c) q.w[i][c] = (float)(w[i][c] / sum[c]);  // odd taps: every sum >= 1
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (taps) {
    case 1: e = launch_ca<1>(q, s); break;
    case 3: e = launch_ca<3>(q, s); break;
    case 5: e = launch_ca<5>(q, s); break;
    case 7: e = launch_ca<7>(q, s); break;
    case 9: e = launch_ca<9>(q, s); break;
    case 11: e = launch_ca<11>(q, s); break;
    case 13: e = launch_ca<13>(q, s); break;
    default: e = launch_ca<15>(q, s); break;
    }
    return e == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}
