// Device-side building blocks of the Wavelet OIT kernels (sm_103a).
//
// One CTA owns one screen tile (<= 256 pixels).  Its fragments are a
// contiguous range of the tile-grouped stream and are read with 16-byte
// vector loads.  Per-pixel state lives in shared memory; fragments of the same
// pixel meet in shared-memory atomics instead of global atomics (the
// coefficient update of §2.3.3).
//
// The build does not touch J+1 coefficients per fragment.  It accumulates two
// per-bin sums per pixel at the finest level (bin m = floor(C z), fraction
// f = C z - m):
//     F_m = sum a_i f_i,      G_m = sum a_i (1 - f_i),
// and turns them into the Haar coefficients of §2.3.1 with an O(C) tree: for
// a dyadic interval I with children L, R and u the position normalised to I,
//     F_I = sum_I a u = (F_L + F_R + S_R)/2,   G_I = sum_I a (1-u) = (S_L + G_L + G_R)/2,
//     sum_I a Psi_{n,k} = 2^{-n/2} (F_L + G_R)/2   (Psi is u, then 1-u, scaled),
// with S = F + G, so X_{n,k} = -2^{-n/2} (F_L + G_R)/2 and chi_00 = G_root.
// Every term is a sum of non-negative numbers, so the FP32 tree adds no
// cancellation.  This is exact algebra on the closed form, not an
// approximation of it.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wt {

constexpr int kThreads = 256;    // threads per CTA
constexpr int kMaxTilePx = 256;  // pixels per tile
// alpha is clamped to [0, 1 - 2^-20] and z to [0, 1 - 2^-24] (exact in FP32)
constexpr float kAlphaMax = 0.99999904632568359375f;
constexpr float kZMax = 0.999999940395355224609375f;
// the largest absorbance step after the clamp: -ln(2^-20) = 20 ln 2
constexpr float kStepCap = 13.8629436111989061f;

struct Geom {
    int width, height, tile_w, tile_h, ntx;
};

// Everything a kernel reads or writes; passed by value.
struct Params {
    Geom g;
    uint32_t flags;
    int64_t n;
    const uint32_t *__restrict__ pixel;
    const float *__restrict__ z;
    const float *__restrict__ alpha;
    const float *__restrict__ r;
    const float *__restrict__ gc;
    const float *__restrict__ b;
    const int64_t *__restrict__ off;
    void *coeff;
    float *zmin;
    float *accum;
    float *out;
    const float *__restrict__ bg_img;
    float bg0, bg1, bg2;
    unsigned long long *err;
};

enum : uint32_t { kSelfExclude = 1u, kLinear = 2u, kNormalized = 4u, kAccumulate = 8u };

// ---------------------------------------------------------------- storage

template <typename T> struct Cvt;
template <> struct Cvt<float> {
    static __device__ __forceinline__ float to(float x) { return x; }
    static __device__ __forceinline__ float from(float x) { return x; }
};
template <> struct Cvt<__nv_bfloat16> {
    static __device__ __forceinline__ __nv_bfloat16 to(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ float from(__nv_bfloat16 x) { return __bfloat162float(x); }
};
template <> struct Cvt<__half> {
    static __device__ __forceinline__ __half to(float x) { return __float2half_rn(x); }
    static __device__ __forceinline__ float from(__half x) { return __half2float(x); }
};
template <typename T> __device__ __forceinline__ float round_to(float x) {
    return Cvt<T>::from(Cvt<T>::to(x));
}

// ---------------------------------------------------------------- tiles

struct Tile {
    int tx0, ty0, tw, th;  // origin and clipped extent
    int64_t s, e;          // fragment range
};

__device__ __forceinline__ Tile tile_of(const Params &p, int t, bool count_bad) {
    Tile T;
    const int tx = t % p.g.ntx, ty = t / p.g.ntx;
    T.tx0 = tx * p.g.tile_w;
    T.ty0 = ty * p.g.tile_h;
    T.tw = min(p.g.tile_w, p.g.width - T.tx0);
    T.th = min(p.g.tile_h, p.g.height - T.ty0);
    int64_t s = p.off[t], e = p.off[t + 1];
    if (s < 0 || e < s || e > p.n) {  // corrupt range: skip the tile, count once
        if (count_bad && threadIdx.x == 0) atomicAdd(p.err, 1ull);
        s = e = 0;
    }
    T.s = s;
    T.e = e;
    return T;
}

// local pixel index inside the tile, or -1 when the pixel is not in it
__device__ __forceinline__ int local_pixel(uint32_t px, const Params &p, const Tile &T) {
    const uint32_t y = px / (uint32_t)p.g.width;
    const uint32_t x = px - y * (uint32_t)p.g.width;
    const int lx = (int)x - T.tx0;
    const int ly = (int)min(y, 0x7fffffffu) - T.ty0;
    if ((unsigned)lx >= (unsigned)T.tw || (unsigned)ly >= (unsigned)T.th) return -1;
    return ly * p.g.tile_w + lx;
}

// ---------------------------------------------------------------- conditioning

__device__ __forceinline__ float clamp_alpha(float al) { return fminf(fmaxf(al, 0.f), kAlphaMax); }
__device__ __forceinline__ float clamp_depth(float z) { return fminf(fmaxf(z, 0.f), kZMax); }
// absorbance step of one interface: v drops by (1 - alpha) across it
__device__ __forceinline__ float step_of(float alpha_c) { return -log1pf(-alpha_c); }

// ---------------------------------------------------------------- streaming

// Calls body(pixel, z, alpha) for every fragment of [s, e), 4 per 16-byte load.
template <class Body>
__device__ __forceinline__ void for_each_frag3(int64_t s, int64_t e, const Params &p, Body &&body) {
    const int tid = threadIdx.x, nt = blockDim.x;
    int64_t s4 = (s + 3) & ~int64_t(3), e4 = e & ~int64_t(3);
    if (s4 > e4) s4 = e4 = e;
    for (int64_t i = s + tid; i < s4; i += nt) body(p.pixel[i], p.z[i], p.alpha[i]);
    const uint4 *px4 = reinterpret_cast<const uint4 *>(p.pixel);
    const float4 *z4 = reinterpret_cast<const float4 *>(p.z);
    const float4 *a4 = reinterpret_cast<const float4 *>(p.alpha);
    for (int64_t q = (s4 >> 2) + tid; q < (e4 >> 2); q += nt) {
        const uint4 pv = px4[q];
        const float4 zv = z4[q];
        const float4 av = a4[q];
        body(pv.x, zv.x, av.x);
        body(pv.y, zv.y, av.y);
        body(pv.z, zv.z, av.z);
        body(pv.w, zv.w, av.w);
    }
    for (int64_t i = e4 + tid; i < e; i += nt) body(p.pixel[i], p.z[i], p.alpha[i]);
}

// Same with colour: body(pixel, z, alpha, r, g, b).
template <class Body>
__device__ __forceinline__ void for_each_frag6(int64_t s, int64_t e, const Params &p, Body &&body) {
    const int tid = threadIdx.x, nt = blockDim.x;
    int64_t s4 = (s + 3) & ~int64_t(3), e4 = e & ~int64_t(3);
    if (s4 > e4) s4 = e4 = e;
    for (int64_t i = s + tid; i < s4; i += nt)
        body(p.pixel[i], p.z[i], p.alpha[i], p.r[i], p.gc[i], p.b[i]);
    const uint4 *px4 = reinterpret_cast<const uint4 *>(p.pixel);
    const float4 *z4 = reinterpret_cast<const float4 *>(p.z);
    const float4 *a4 = reinterpret_cast<const float4 *>(p.alpha);
    const float4 *r4 = reinterpret_cast<const float4 *>(p.r);
    const float4 *g4 = reinterpret_cast<const float4 *>(p.gc);
    const float4 *b4 = reinterpret_cast<const float4 *>(p.b);
    for (int64_t q = (s4 >> 2) + tid; q < (e4 >> 2); q += nt) {
        const uint4 pv = px4[q];
        const float4 zv = z4[q], av = a4[q], rv = r4[q], gv = g4[q], bv = b4[q];
        body(pv.x, zv.x, av.x, rv.x, gv.x, bv.x);
        body(pv.y, zv.y, av.y, rv.y, gv.y, bv.y);
        body(pv.z, zv.z, av.z, rv.z, gv.z, bv.z);
        body(pv.w, zv.w, av.w, rv.w, gv.w, bv.w);
    }
    for (int64_t i = e4 + tid; i < e; i += nt)
        body(p.pixel[i], p.z[i], p.alpha[i], p.r[i], p.gc[i], p.b[i]);
}

// ---------------------------------------------------------------- error count

__device__ __forceinline__ void flush_bad(unsigned bad, unsigned long long *err) {
    bad = __reduce_add_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(err, (unsigned long long)bad);
}

// ---------------------------------------------------------------- phases

template <int J> struct Shape {
    static constexpr int C = 1 << J;
    static constexpr int LD = C + 1;  // padded row: thread-per-pixel access is conflict free
};

__device__ __forceinline__ void fill_smem(float *a, int count, float v) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) a[i] = v;
}

// Step 2 accumulation: per fragment, 2 shared-memory adds into its bin.
template <int J>
__device__ __forceinline__ void phase_bins(const Params &p, const Tile &T, float *sF, float *sG,
                                           unsigned *sZ, unsigned &bad) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD;
    for_each_frag3(T.s, T.e, p, [&](uint32_t px, float z, float al) {
        if (!(z == z) || !(al == al)) {
            ++bad;
            return;
        }
        const int lp = local_pixel(px, p, T);
        if (lp < 0) {
            ++bad;
            return;
        }
        const float a = step_of(clamp_alpha(al));
        const float zc = clamp_depth(z);
        const float s = zc * (float)C;  // exact: C is a power of two
        const int m = (int)s;
        const float f = s - (float)m;
        atomicAdd(&sF[lp * LD + m], a * f);
        atomicAdd(&sG[lp * LD + m], a * (1.f - f));
        const unsigned zb = __float_as_uint(zc);
        if (a > 0.f && zb < sZ[lp]) atomicMin(&sZ[lp], zb);
    });
}

// 2^{n/2} and 2^{-n/2}/2 as compile-time constants
__device__ __forceinline__ constexpr float sqrt2_pow(int n) {
    return (n & 1 ? 1.41421356237309505f : 1.f) * (float)(1u << (n >> 1));
}
__device__ __forceinline__ constexpr float half_inv_sqrt2_pow(int n) {
    return 0.5f / sqrt2_pow(n);
}

// Bins (F, G) -> Haar coefficients in heap order, in place in sF.
// C lanes per pixel (C <= 32), one shuffle tree per pixel.
template <int J>
__device__ __forceinline__ void phase_bins_to_coeffs(float *sF, const float *sG, int npx) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD, PPW = 32 / C;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int seg = lane / C, m = lane % C;
    for (int p0 = warp * PPW; p0 < npx; p0 += nwarps * PPW) {
        const int px = p0 + seg;
        const bool live = px < npx;
        float F = live ? sF[px * LD + m] : 0.f;
        float G = live ? sG[px * LD + m] : 0.f;
        __syncwarp();
#pragma unroll
        for (int n = J - 1; n >= 0; --n) {
            const int d = 1 << (J - 1 - n);  // lane distance between the two children
            const float FR = __shfl_down_sync(0xffffffffu, F, d, C);
            const float GR = __shfl_down_sync(0xffffffffu, G, d, C);
            const float coef = -half_inv_sqrt2_pow(n) * (F + GR);
            const float Fp = 0.5f * ((F + FR) + (FR + GR));
            const float Gp = 0.5f * ((F + G) + (G + GR));
            if (live && (m & (2 * d - 1)) == 0) sF[px * LD + (1 << n) + m / (2 * d)] = coef;
            F = Fp;
            G = Gp;
        }
        if (live && m == 0) sF[px * LD] = G;
        __syncwarp();
    }
}

// Haar synthesis at the bin centres, in place:
// A_m = chi_00 + sum_n +-2^{n/2} X_{n, m>>(J-n)} (+ in the first half of psi's support).
template <int J>
__device__ __forceinline__ void phase_coeffs_to_bins(float *sC, int npx) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD, PPW = 32 / C;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int seg = lane / C, m = lane % C;
    for (int p0 = warp * PPW; p0 < npx; p0 += nwarps * PPW) {
        const int px = p0 + seg;
        float A = 0.f;
        if (px < npx) {
            const float *c = sC + px * LD;
            A = c[0];
#pragma unroll
            for (int n = 0; n < J; ++n) {
                const float d = sqrt2_pow(n) * c[(1 << n) + (m >> (J - n))];
                A += ((m >> (J - 1 - n)) & 1) ? -d : d;
            }
        }
        __syncwarp();
        if (px < npx) sC[px * LD + m] = A;
        __syncwarp();
    }
}

// Reconstruction at (m, f) from bin values, and the fragment's own step there.
// Linear: interpolate between bin centres; constant in the two outer half-bins.
template <int J>
__device__ __forceinline__ float recon(const float *A, int m, float f, uint32_t flags,
                                       float a, float &self) {
    constexpr int C = Shape<J>::C;
    if (!(flags & kLinear)) {
        self = a * (1.f - f);
        return A[m];
    }
    if (f < 0.5f) {
        if (m == 0) {
            self = a * (1.f - f);
            return A[0];
        }
        const float t = f + 0.5f;
        self = a * (1.f - f) * t;
        return fmaf(t, A[m] - A[m - 1], A[m - 1]);
    }
    if (m == C - 1) {
        self = a * (1.f - f);
        return A[C - 1];
    }
    const float t = f - 0.5f;
    self = a * fmaf(1.f - f, 1.f - t, t);
    return fmaf(t, A[m + 1] - A[m], A[m]);
}

// Absorbance in front of a fragment (§2.3.2 with the self term removed).
template <int J>
__device__ __forceinline__ float frag_absorbance(const float *A, float zc, float a, uint32_t flags) {
    constexpr int C = Shape<J>::C;
    const float s = zc * (float)C;
    const int m = (int)s;
    const float f = s - (float)m;
    float self;
    const float full = recon<J>(A, m, f, flags, a, self);
    return (flags & kSelfExclude) ? fmaxf(full - self, 0.f) : full;
}

// Per-pixel weight offset m_p: every fragment's absorbance is >= m_p and the
// nearest one's is <= m_p + kStepCap, so exp(m_p - A_i) never overflows and
// the largest weight never underflows.
template <int J>
__device__ __forceinline__ float weight_offset(const float *A, float zmin, uint32_t flags) {
    if (!(zmin < 1.f)) return 0.f;  // +inf: no fragment with alpha > 0
    const float full = frag_absorbance<J>(A, clamp_depth(zmin), 0.f, flags & kLinear);
    return fmaxf(full - kStepCap, 0.f);
}

// Step 3 (§2.1): per fragment v_i = exp(-A_i), w_i = alpha_i v_i; per pixel
// R,G,B += c_i w_i, W += w_i, S += a_i (five shared-memory adds).  Weights
// carry the pixel's offset m_p: w_i' = alpha_i exp(m_p - A_i).
template <int J, bool COUNT>
__device__ __forceinline__ void phase_resolve(const Params &p, const Tile &T, const float *sA,
                                              const float *sMp, float *sAcc, int npx,
                                              unsigned &bad) {
    constexpr int LD = Shape<J>::LD;
    const uint32_t flags = p.flags;
    for_each_frag6(T.s, T.e, p, [&](uint32_t px, float z, float al, float r, float g, float b) {
        if (!(z == z) || !(al == al)) {
            if (COUNT) ++bad;
            return;
        }
        const int lp = local_pixel(px, p, T);
        if (lp < 0) {
            if (COUNT) ++bad;
            return;
        }
        const float ac = clamp_alpha(al);
        const float a = step_of(ac);
        const float Ah = frag_absorbance<J>(sA + lp * LD, clamp_depth(z), a, flags);
        const float w = ac * expf(sMp[lp] - Ah);
        atomicAdd(&sAcc[lp], r * w);
        atomicAdd(&sAcc[npx + lp], g * w);
        atomicAdd(&sAcc[2 * npx + lp], b * w);
        atomicAdd(&sAcc[3 * npx + lp], w);
        atomicAdd(&sAcc[4 * npx + lp], a);
    });
}

// global pixel id of local pixel lp, or -1 if it lies outside the image
__device__ __forceinline__ int64_t global_pixel(const Params &p, const Tile &T, int lp) {
    const int lx = lp % p.g.tile_w, ly = lp / p.g.tile_w;
    if (lx >= T.tw || ly >= T.th) return -1;
    return (int64_t)(T.ty0 + ly) * p.g.width + T.tx0 + lx;
}

// Step 4 (§2.1): composite one pixel over the background.
__device__ __forceinline__ void composite_pixel(const Params &p, int64_t gp, float R, float G,
                                                float B, float W, float S) {
    float bg0 = p.bg0, bg1 = p.bg1, bg2 = p.bg2;
    if (p.bg_img) {
        bg0 = p.bg_img[3 * gp];
        bg1 = p.bg_img[3 * gp + 1];
        bg2 = p.bg_img[3 * gp + 2];
    }
    const float T = expf(-S);
    const float cover = -expm1f(-S);  // 1 - T without cancellation
    float4 o;
    if (p.flags & kNormalized) {
        if (W > 0.f) {
            const float k = cover / W;
            o.x = fmaf(R, k, bg0 * T);
            o.y = fmaf(G, k, bg1 * T);
            o.z = fmaf(B, k, bg2 * T);
        } else {
            o.x = bg0;
            o.y = bg1;
            o.z = bg2;
        }
    } else {
        o.x = fmaf(bg0, T, R);
        o.y = fmaf(bg1, T, G);
        o.z = fmaf(bg2, T, B);
    }
    o.w = cover;
    reinterpret_cast<float4 *>(p.out)[gp] = o;
}

// Epilogue of the resolve: composite into out, or write/add accum.
template <bool COMPOSITE>
__device__ __forceinline__ void resolve_epilogue(const Params &p, const Tile &T, const float *sAcc,
                                                 int npx) {
    for (int lp = threadIdx.x; lp < npx; lp += blockDim.x) {
        const int64_t gp = global_pixel(p, T, lp);
        if (gp < 0) continue;
        const float R = sAcc[lp], G = sAcc[npx + lp], B = sAcc[2 * npx + lp];
        const float W = sAcc[3 * npx + lp], S = sAcc[4 * npx + lp];
        if (COMPOSITE) {
            composite_pixel(p, gp, R, G, B, W, S);
        } else {
            float *acc = p.accum + 5 * gp;
            if (p.flags & kAccumulate) {
                acc[0] += R;
                acc[1] += G;
                acc[2] += B;
                acc[3] += W;
                acc[4] += S;
            } else {
                acc[0] = R;
                acc[1] = G;
                acc[2] = B;
                acc[3] = W;
                acc[4] = S;
            }
        }
    }
}

// Coalesced tile <-> coefficient buffer copies.  Row ly of a tile is a
// contiguous run of tw*C coefficients in the pixel-major buffer.
template <int J, typename CT>
__device__ __forceinline__ void load_coeffs(const Params &p, const Tile &T, float *sC) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD;
    const CT *src = static_cast<const CT *>(p.coeff);
    const int rowlen = T.tw * C;
    for (int ly = 0; ly < T.th; ++ly) {
        const int64_t base = ((int64_t)(T.ty0 + ly) * p.g.width + T.tx0) * C;
        for (int e = threadIdx.x; e < rowlen; e += blockDim.x)
            sC[(ly * p.g.tile_w + (e >> J)) * LD + (e & (C - 1))] = Cvt<CT>::from(src[base + e]);
    }
}

// Rounds the tile's coefficients to the storage type in place and, when
// `store`, writes them (adding the stored values first when `accumulate`).
template <int J, typename CT>
__device__ __forceinline__ void round_store_coeffs(const Params &p, const Tile &T, float *sC,
                                                   bool store, bool accumulate) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD;
    CT *dst = static_cast<CT *>(p.coeff);
    const int rowlen = T.tw * C;
    for (int ly = 0; ly < T.th; ++ly) {
        const int64_t base = ((int64_t)(T.ty0 + ly) * p.g.width + T.tx0) * C;
        for (int e = threadIdx.x; e < rowlen; e += blockDim.x) {
            float *slot = &sC[(ly * p.g.tile_w + (e >> J)) * LD + (e & (C - 1))];
            float v = *slot;
            if (accumulate) v += Cvt<CT>::from(dst[base + e]);
            const CT q = Cvt<CT>::to(v);
            *slot = Cvt<CT>::from(q);
            if (store) dst[base + e] = q;
        }
    }
}

__device__ __forceinline__ void store_zmin(const Params &p, const Tile &T, const unsigned *sZ,
                                           int npx, bool accumulate) {
    for (int lp = threadIdx.x; lp < npx; lp += blockDim.x) {
        const int64_t gp = global_pixel(p, T, lp);
        if (gp < 0) continue;
        float v = __uint_as_float(sZ[lp]);
        if (accumulate) v = fminf(v, p.zmin[gp]);
        p.zmin[gp] = v;
    }
}

// Shared-memory footprints (floats), shared by kernels and launchers.
template <int J> struct Smem {
    // build / fused: F and G rows + nearest-depth word per pixel
    static constexpr size_t bins(int npx) { return (size_t)(2 * npx * Shape<J>::LD + npx); }
    // resolve: coefficient/bin rows + m_p + 5 accumulators per pixel
    static constexpr size_t resolve(int npx) { return (size_t)(npx * Shape<J>::LD + 6 * npx); }
};

}  // namespace wt
