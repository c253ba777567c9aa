// Coloured absorbance: the three-channel form of the method (§1.2: the
// visibility function may differ per colour; §2.1: the paper's coefficients
// carry three channels, packed E5B9G9R9).  Fragment i has one depth and one
// opacity per channel, alpha_c; channel c has its own absorbance steps
// a_c = -ln(1 - alpha_c), its own Haar coefficients, its own transmittance
// v_c = exp(-A_c) and its own normalised resolve
//     out_c = (R_c / W_c)(1 - T_c) + bg_c T_c,  R_c = sum col_c alpha_c v_c,
//     W_c = sum alpha_c v_c,  T_c = exp(-sum a_c),
// so each channel is the mono method on (z, alpha_c, col_c).
//
// One fused tile kernel builds the three channels' bins in one pass over the
// fragments (six fixed-point planes), turns them into coefficients, rounds
// them through the storage format (FP32, or the E5B9G9R9 triple of each
// coefficient index), synthesises three rows of bin values and resolves the
// three channels in a second pass, the coefficients never leaving the SM.
#include "wt.h"
#include "wt_internal.h"
#include "wt_tile.cuh"

namespace wt {

unsigned long long *error_word();  // wt_api.cu

namespace {

constexpr int kCh = 3;

struct RgbParams {
    Params p;  // geometry, fragments (pixel, z, r, g, b), coeff (nullable), out, bg, err
    const float *__restrict__ alpha_c[kCh];
    int e5;  // storage: 1 = E5B9G9R9 [P][C] words, 0 = FP32 [P][3][C]
};

template <int J> struct RgbLayout {
    static constexpr size_t plane(int npx) { return Layout<J>::plane(npx); }
    static constexpr size_t vplane(int npx) { return Layout<J>::vplane(npx); }
    static constexpr size_t accw(int npx) { return (size_t)kWarps * npx * 32; }  // 2 float4 per pixel
    static constexpr size_t words(int npx) { return Layout<J>::words(npx); }
    static constexpr size_t build(int npx) { return 2 * kCh * plane(npx); }
    static constexpr size_t resolve(int npx) { return kCh * vplane(npx) + accw(npx) + kCh * words(npx); }
    static constexpr size_t region(int npx) { return build(npx) > resolve(npx) ? build(npx) : resolve(npx); }
    static constexpr size_t total(int npx) { return region(npx) + words(npx); }  // + nearest-depth words
};

// Warp-segmented reduction of eight floats per pixel (the rank rounds of
// warp_accumulate, on two float4 halves).
__device__ __forceinline__ void accumulate8(float4 *mine, int lp, float4 v0, float4 v1) {
    float4 o0 = mine[2 * lp], o1 = mine[2 * lp + 1];
    o0.x += v0.x, o0.y += v0.y, o0.z += v0.z, o0.w += v0.w;
    o1.x += v1.x, o1.y += v1.y, o1.z += v1.z, o1.w += v1.w;
    mine[2 * lp] = o0;
    mine[2 * lp + 1] = o1;
}
__device__ __forceinline__ void warp_accumulate8(float4 *mine, int lp, float4 v0, float4 v1) {
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    const unsigned rank = __popc(__match_any_sync(0xffffffffu, lp) & lt);
    if (lp >= 0 && rank == 0) accumulate8(mine, lp, v0, v1);
    __syncwarp();
    for (unsigned r = 1; __any_sync(0xffffffffu, lp >= 0 && rank >= r); ++r) {
        if (lp >= 0 && rank == r) accumulate8(mine, lp, v0, v1);
        __syncwarp();
    }
}

// Counting pass of the fallback for three channels: per pixel the fragment
// count and the largest clamped opacity over the channels, then one scale s_p
// for all three channels' bins.
template <int J>
__device__ __forceinline__ void count_pass_rgb(const RgbParams &q, const Tile &T, unsigned *sF0) {
    constexpr int LD = Shape<J>::LD;
    constexpr int CNT = Shape<J>::CNT, AMAX = Shape<J>::AMAX, INV = Shape<J>::INV;
    const Params &p = q.p;
    for (int64_t i = T.s + threadIdx.x; i < T.e; i += blockDim.x) {
        const float z = p.z[i];
        float am = 0.f;
        bool nan = !(z == z);
#pragma unroll
        for (int c = 0; c < kCh; ++c) {
            const float al = q.alpha_c[c][i];
            nan |= !(al == al);
            am = fmaxf(am, clamp_alpha(al));
        }
        const int lp = nan ? -1 : local_pixel(p.pixel[i], p, T);
        if (lp >= 0) {
            atomicAdd(&sF0[lp * LD + CNT], 1u);
            atomicMax(&sF0[lp * LD + AMAX], __float_as_uint(am));
        }
    }
    __syncthreads();
    for (int lp = threadIdx.x; lp < p.g.tile_w * p.g.tile_h; lp += blockDim.x) {
        unsigned *row = sF0 + lp * LD;
        const float bound = (float)row[CNT] * step_of(__uint_as_float(row[AMAX]));
        const int e = bound > 0.f ? max(ilogbf(bound), -30) : 0;
        row[INV] = __float_as_uint(ldexpf(1.f, e - 30));
        row[AMAX] = __float_as_uint(ldexpf(1.f, 30 - e));
    }
    __syncthreads();
}

// Bins of the three channels: fixed scale 2^27 (SCALED = false, reports a
// wrapped word or a step below 2^-7) or the per-pixel scale of channel 0's row
// (SCALED = true).  Plane 2c is channel c's F, plane 2c+1 its G.
template <int J, bool SCALED, bool COUNT>
__device__ __forceinline__ bool bins_pass_rgb(const RgbParams &q, const Tile &T, unsigned *planes, size_t pl,
                                              unsigned *sZ, unsigned &bad) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD, AMAX = Shape<J>::AMAX;
    constexpr float kFineStep = 1048576.f;  // 2^20: a step of 2^-7 under the fixed scale
    const Params &p = q.p;
    bool retry = false;
    for (int64_t i = T.s + threadIdx.x; i < T.e; i += blockDim.x) {
        const float z = p.z[i];
        float al[kCh];
        bool nan = !(z == z);
#pragma unroll
        for (int c = 0; c < kCh; ++c) {
            al[c] = q.alpha_c[c][i];
            nan |= !(al[c] == al[c]);
        }
        const int lp = nan ? -1 : local_pixel(p.pixel[i], p, T);
        if (lp < 0) {
            if (COUNT) ++bad;
            continue;
        }
        const float zc = clamp_depth(z);
        const float s = zc * (float)C;
        const Floor m = floor_small(s);
        const float f = s - m.f;
        const float sp = SCALED ? __uint_as_float(planes[lp * LD + AMAX]) : kBinScale;
        bool any = false;
#pragma unroll
        for (int c = 0; c < kCh; ++c) {
            const float a = step_of(clamp_alpha(al[c]));
            const float as = a * sp;
            const unsigned vF = __float2uint_rn(as * f), vG = __float2uint_rn(as * (1.f - f));
            unsigned *F = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(planes) + (2 * c) * pl);
            unsigned *G = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(planes) + (2 * c + 1) * pl);
            const unsigned oF = atomicAdd(&F[lp * LD + m.i], vF);
            const unsigned oG = atomicAdd(&G[lp * LD + m.i], vG);
            if (!SCALED) retry |= (oF + vF < oF) | (oG + vG < oG) | (as < kFineStep && a > 0.f);
            any |= a > 0.f;
        }
        if (any) atomicMin(&sZ[lp], __float_as_uint(zc));
    }
    return retry;
}

template <int J>
__global__ void __launch_bounds__(kThreads, 2) k_fused_rgb(RgbParams q) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD, LDV = Shape<J>::LDV;
    extern __shared__ __align__(16) unsigned char smem[];
    const Params &p = q.p;
    const int npx = p.g.tile_w * p.g.tile_h;
    const size_t pl = RgbLayout<J>::plane(npx), vpl = RgbLayout<J>::vplane(npx), wd = RgbLayout<J>::words(npx);
    unsigned *planes = reinterpret_cast<unsigned *>(smem);  // 6 bins planes, later 3 value planes
    float *vals = reinterpret_cast<float *>(smem);
    float4 *accw = reinterpret_cast<float4 *>(smem + kCh * vpl);
    float *sS = reinterpret_cast<float *>(smem + kCh * vpl + RgbLayout<J>::accw(npx));  // 3 word planes
    unsigned *sZ = reinterpret_cast<unsigned *>(smem + RgbLayout<J>::region(npx));
    const Tile T = tile_of(p, p.tile0 + (int)blockIdx.x, true);
    fill_zero(smem, (int)(2 * kCh * pl));
    for (int i = threadIdx.x; i < npx; i += blockDim.x) sZ[i] = 0x7f800000u;
    __syncthreads();
    unsigned bad = 0;
    const bool retry = bins_pass_rgb<J, false, true>(q, T, planes, pl, sZ, bad);
    flush_bad(bad, p.err);
    const bool scaled = __syncthreads_or(retry);
    if (scaled) {
        fill_zero(smem, (int)(2 * kCh * pl));
        __syncthreads();
        count_pass_rgb<J>(q, T, planes);
        bins_pass_rgb<J, true, false>(q, T, planes, pl, sZ, bad);
        __syncthreads();
    }
    const int lp = threadIdx.x;
    int64_t gp = -1;
    if (lp < npx) gp = global_pixel(p, T, lp);
    // coefficients of the three channels, rounded through the storage format
    float co[kCh][C], S[kCh] = {0.f, 0.f, 0.f};
    if (gp >= 0) {
        // one scale for all three channels: 2^-27, or channel 0's row's 1 / s_p
        const float inv = scaled ? __uint_as_float(planes[lp * LD + Shape<J>::INV]) : kBinInv;
#pragma unroll
        for (int c = 0; c < kCh; ++c) {
            const unsigned *F = reinterpret_cast<const unsigned *>(smem + 2 * c * pl);
            const unsigned *G = reinterpret_cast<const unsigned *>(smem + (2 * c + 1) * pl);
            bins_to_coeffs_inv<J>(F + lp * LD, G + lp * LD, inv, co[c], S[c]);
        }
        if (q.e5) {
            // E5B9G9R9 of each coefficient index (magnitudes: chi >= 0, X <= 0)
#pragma unroll
            for (int k = 0; k < C; ++k) {
                const float sg = k == 0 ? 1.f : -1.f;
                const uint32_t w = e5_encode(sg * co[0][k], sg * co[1][k], sg * co[2][k]);
                if (p.coeff) static_cast<uint32_t *>(p.coeff)[gp * C + k] = w;
                float r, g, b;
                e5_decode(w, r, g, b);
                co[0][k] = sg * r;
                co[1][k] = sg * g;
                co[2][k] = sg * b;
            }
        } else if (p.coeff) {
            float *dst = static_cast<float *>(p.coeff) + gp * kCh * C;
#pragma unroll
            for (int c = 0; c < kCh; ++c) store_row<float, C>(dst + c * C, co[c]);
        }
    }
    __syncthreads();  // every bin row has been read
    if (gp >= 0) {
#pragma unroll
        for (int c = 0; c < kCh; ++c) {
            coeffs_to_bins<J>(co[c], kLog2e);
            put_bins<J>(reinterpret_cast<float *>(reinterpret_cast<char *>(vals) + c * vpl) + lp * LDV, co[c],
                        __uint_as_float(sZ[lp]), p.flags);
            sS[c * (wd / 4) + lp] = S[c];
        }
    }
    fill_zero(accw, (int)RgbLayout<J>::accw(npx));
    __syncthreads();
    // resolve the three channels
    const uint32_t flags = p.flags;
    float4 *mine = accw + (threadIdx.x >> 5) * 2 * npx;
    const int nt = blockDim.x;
    const int64_t rounds = (T.e - T.s + nt - 1) / nt;  // equal trip counts: warp collectives below
    for (int64_t it = 0; it < rounds; ++it) {
        const int64_t i = T.s + it * nt + threadIdx.x;
        const bool v = i < T.e;
        int l = -1;
        float w[kCh] = {0.f, 0.f, 0.f}, col[kCh] = {0.f, 0.f, 0.f};
        if (v) {
            const float z = p.z[i];
            float al[kCh];
            bool nan = !(z == z);
#pragma unroll
            for (int c = 0; c < kCh; ++c) {
                al[c] = q.alpha_c[c][i];
                nan |= !(al[c] == al[c]);
            }
            l = nan ? -1 : local_pixel(p.pixel[i], p, T);
            if (l >= 0) {
                col[0] = p.r[i];
                col[1] = p.gc[i];
                col[2] = p.b[i];
                const float zc = clamp_depth(z);
#pragma unroll
                for (int c = 0; c < kCh; ++c) {
                    const float ac = clamp_alpha(al[c]);
                    const float *row =
                        reinterpret_cast<const float *>(reinterpret_cast<const char *>(vals) + c * vpl) + l * LDV;
                    const float Ah = absorbance_at<J>(row, zc, -lg2(1.f - ac), flags);
                    w[c] = ac * ex2(-Ah);
                }
            }
        }
        warp_accumulate8(mine, l, make_float4(col[0] * w[0], col[1] * w[1], col[2] * w[2], w[0]),
                         make_float4(w[1], w[2], 0.f, 0.f));
    }
    __syncthreads();
    if (gp >= 0) {
        float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
        for (int wp = 0; wp < kWarps; ++wp) {
            const float4 u0 = accw[wp * 2 * npx + 2 * lp], u1 = accw[wp * 2 * npx + 2 * lp + 1];
            a0.x += u0.x, a0.y += u0.y, a0.z += u0.z, a0.w += u0.w;
            a1.x += u1.x, a1.y += u1.y;
        }
        const float R[kCh] = {a0.x, a0.y, a0.z}, W[kCh] = {a0.w, a1.x, a1.y};
        const float bg[kCh] = {p.bg_img ? p.bg_img[3 * gp] : p.bg0, p.bg_img ? p.bg_img[3 * gp + 1] : p.bg1,
                               p.bg_img ? p.bg_img[3 * gp + 2] : p.bg2};
        float o[kCh], cover_sum = 0.f;
#pragma unroll
        for (int c = 0; c < kCh; ++c) {
            const float Sc = sS[c * (wd / 4) + lp];
            const float Tc = ex2(-Sc * kLog2e);
            const float cover = Sc < 0.0009765625f ? Sc * fmaf(-0.5f, Sc, 1.f) : 1.f - Tc;
            cover_sum += cover;
            if (flags & kNormalized) {
                o[c] = W[c] > 0.f ? fmaf(R[c], cover / W[c], bg[c] * Tc) : bg[c];
            } else {
                o[c] = fmaf(bg[c], Tc, R[c]);
            }
        }
        reinterpret_cast<float4 *>(p.out)[gp] = make_float4(o[0], o[1], o[2], cover_sum * (1.f / 3.f));
    }
}

template <int J> cudaError_t launch_rgb(const RgbParams &q, int ntiles, cudaStream_t s) {
    const int npx = q.p.g.tile_w * q.p.g.tile_h;
    const size_t bytes = RgbLayout<J>::total(npx);
    if (bytes > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_fused_rgb<J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_fused_rgb<J><<<ntiles, kThreads, bytes, s>>>(q);
    return cudaGetLastError();
}

typedef cudaError_t (*RgbLaunch)(const RgbParams &, int, cudaStream_t);
const RgbLaunch kRgb[5] = {launch_rgb<1>, launch_rgb<2>, launch_rgb<3>, launch_rgb<4>, launch_rgb<5>};

}  // namespace

// Shared memory the coloured kernel needs for a tile of npx pixels at J.
size_t rgb_smem_bytes(int J, int npx) {
    switch (J) {
    case 1: return RgbLayout<1>::total(npx);
    case 2: return RgbLayout<2>::total(npx);
    case 3: return RgbLayout<3>::total(npx);
    case 4: return RgbLayout<4>::total(npx);
    default: return RgbLayout<5>::total(npx);
    }
}

cudaError_t launch_fused_rgb(const Params &p, int J, const float *const alpha_c[3], bool e5, int ntiles,
                             cudaStream_t s) {
    RgbParams q;
    q.p = p;
    for (int c = 0; c < kCh; ++c) q.alpha_c[c] = alpha_c[c];
    q.e5 = e5 ? 1 : 0;
    return kRgb[J - 1](q, ntiles, s);
}

}  // namespace wt
