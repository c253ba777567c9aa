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
// One thread per pixel; the background is read through the read-only path and
// the neighbouring pixels' taps hit the same lines.
#include <math.h>

#include "wt.h"
#include "wt_internal.h"
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

// Bilinear sample of the RGB background at (x, y) (texel (i, j) centred at
// (i + 1/2, j + 1/2)), clamped to the edge.  Coordinates far outside the image
// are clamped before the integer conversion.
__device__ __forceinline__ float3 bilinear(const CaParams &q, float x, float y) {
    const float fx = x - 0.5f, fy = y - 0.5f;
    float x0 = floorf(fx), y0 = floorf(fy);
    const float ax = fx - x0, ay = fy - y0;
    x0 = fminf(fmaxf(x0, -1.f), (float)q.width);
    y0 = fminf(fmaxf(y0, -1.f), (float)q.height);
    const int ia = (int)x0, ja = (int)y0;
    const int i0 = min(max(ia, 0), q.width - 1), i1 = min(max(ia + 1, 0), q.width - 1);
    const int j0 = min(max(ja, 0), q.height - 1), j1 = min(max(ja + 1, 0), q.height - 1);
    const float *r0 = q.bg + 3 * (int64_t)j0 * q.width, *r1 = q.bg + 3 * (int64_t)j1 * q.width;
    const float w00 = (1.f - ax) * (1.f - ay), w10 = ax * (1.f - ay), w01 = (1.f - ax) * ay, w11 = ax * ay;
    float3 v;
    v.x = w00 * __ldg(r0 + 3 * i0) + w10 * __ldg(r0 + 3 * i1) + w01 * __ldg(r1 + 3 * i0) + w11 * __ldg(r1 + 3 * i1);
    v.y = w00 * __ldg(r0 + 3 * i0 + 1) + w10 * __ldg(r0 + 3 * i1 + 1) + w01 * __ldg(r1 + 3 * i0 + 1) +
          w11 * __ldg(r1 + 3 * i1 + 1);
    v.z = w00 * __ldg(r0 + 3 * i0 + 2) + w10 * __ldg(r0 + 3 * i1 + 2) + w01 * __ldg(r1 + 3 * i0 + 2) +
          w11 * __ldg(r1 + 3 * i1 + 2);
    return v;
}

template <int TAPS> __global__ void __launch_bounds__(256) k_composite_ca(CaParams q) {
    const int64_t P = (int64_t)q.width * q.height;
    unsigned bad = 0;
    for (int64_t gp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gp < P; gp += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(gp / q.width), x = (int)(gp - (int64_t)y * q.width);
        float2 d = q.offset ? q.offset[gp] : make_float2(0.f, 0.f);
        if (!(fabsf(d.x) <= 3.4e38f) || !(fabsf(d.y) <= 3.4e38f)) {  // NaN or infinite: no shift
            d = make_float2(0.f, 0.f);
            ++bad;
        }
        const float cx = (float)x + 0.5f, cy = (float)y + 0.5f;
        float3 bgc = make_float3(0.f, 0.f, 0.f);
#pragma unroll
        for (int i = 0; i < TAPS; ++i) {
            const float3 v = bilinear(q, fmaf(q.s[i], d.x, cx), fmaf(q.s[i], d.y, cy));
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
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t P = (int64_t)q.width * q.height;
    const int64_t want = (P + 255) / 256, cap = (int64_t)sms * 8;
    k_composite_ca<TAPS><<<(int)(want < cap ? want : cap), 256, 0, s>>>(q);
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
    if (!desc || desc->width < 1 || desc->height < 1 || desc->reserved != 0) return WT_ERR_ARG;
    if ((int64_t)desc->width * desc->height >= (int64_t(1) << 31)) return WT_ERR_ARG;
    if (!accum || (reinterpret_cast<uintptr_t>(accum) & 3) || !bg_img || (reinterpret_cast<uintptr_t>(bg_img) & 3))
        return WT_ERR_ARG;
    if ((offset && (reinterpret_cast<uintptr_t>(offset) & 7)) || !out || (reinterpret_cast<uintptr_t>(out) & 15))
        return WT_ERR_ARG;
    if (taps < 1 || taps > kMaxTaps || taps % 2 == 0) return WT_ERR_ARG;
    if (!(dispersion >= 0.f) || !(dispersion <= 3.4e38f)) return WT_ERR_ARG;
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
