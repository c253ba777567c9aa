// Kernels of the Wavelet OIT hot path.  One CTA per screen tile, 256 threads.
// Instantiated per J (1..5) and coefficient storage type in wt_kernels_*.cu.
#pragma once

#include "wt_internal.h"
#include "wt_tile.cuh"

namespace wt {

// Blocks per SM the kernels are compiled for (caps registers per thread so
// that shared memory, not registers, sets the occupancy).
template <int J> struct MinBlocks { static constexpr int value = J >= 5 ? 3 : 4; };

// §2.1 step 2: build the tile's coefficients and store them once.
template <int J, typename CT>
__global__ void __launch_bounds__(kThreads, MinBlocks<J>::value) k_build(Params p) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD;
    extern __shared__ __align__(16) unsigned char smem[];
    const int npx = p.g.tile_w * p.g.tile_h;
    float *sF = reinterpret_cast<float *>(smem);
    float *sG = reinterpret_cast<float *>(smem + Layout<J>::plane(npx));
    unsigned *sZ = reinterpret_cast<unsigned *>(smem + 2 * Layout<J>::plane(npx));
    const Tile T = tile_of(p, blockIdx.x, true);
    fill_zero(smem, (int)(2 * Layout<J>::plane(npx)));
    for (int i = threadIdx.x; i < npx; i += blockDim.x) sZ[i] = 0x7f800000u;  // +inf
    __syncthreads();
    unsigned bad = 0;
    phase_bins<J>(p, T, sF, sG, sZ, bad);
    flush_bad(bad, p.err);
    __syncthreads();
    const int lp = threadIdx.x;
    if (lp >= npx) return;
    const int64_t gp = global_pixel(p, T, lp);
    if (gp < 0) return;
    float c[C], S;
    bins_to_coeffs<J>(sF + lp * LD, sG + lp * LD, c, S);
    CT *dst = static_cast<CT *>(p.coeff) + gp * C;
    const bool acc = (p.flags & kAccumulate) != 0;
    if (acc) {
        float old[C];
        load_row<CT, C>(dst, old);
#pragma unroll
        for (int i = 0; i < C; ++i) c[i] += old[i];
    }
    store_row<CT, C>(dst, c);
    if (p.zmin) {
        float v = __uint_as_float(sZ[lp]);
        if (acc) v = fminf(v, p.zmin[gp]);
        p.zmin[gp] = v;
    }
}

// Writes one pixel's bin values (log2 units) into its shared row.
template <int J> __device__ __forceinline__ void put_vals(float *row, const float (&v)[1 << J]) {
    constexpr int C = 1 << J;
    if constexpr (C % 4 == 0) {
#pragma unroll
        for (int q = 0; q < C / 4; ++q)
            reinterpret_cast<float4 *>(row)[q] =
                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < C; ++i) row[i] = v[i];
    }
}

// §2.1 step 3 (+ step 4 when COMPOSITE): resolve against stored coefficients.
template <int J, typename CT, bool COMPOSITE>
__global__ void __launch_bounds__(kThreads, MinBlocks<J>::value) k_resolve(Params p) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD;
    extern __shared__ __align__(16) unsigned char smem[];
    const int npx = p.g.tile_w * p.g.tile_h;
    float *vals = reinterpret_cast<float *>(smem);
    float *acc = reinterpret_cast<float *>(smem + Layout<J>::plane(npx));
    float *sMp = reinterpret_cast<float *>(smem + Layout<J>::plane(npx) + Layout<J>::acc(npx, 5));
    const Tile T = tile_of(p, blockIdx.x, true);
    const int lp = threadIdx.x;
    int64_t gp = -1;
    if (lp < npx) gp = global_pixel(p, T, lp);
    if (gp >= 0) {
        float v[C];
        load_row<CT, C>(static_cast<const CT *>(p.coeff) + gp * C, v);
        coeffs_to_bins<J>(v);
#pragma unroll
        for (int i = 0; i < C; ++i) v[i] *= kLog2e;
        put_vals<J>(vals + lp * LD, v);
        const bool use_offset = (p.flags & kNormalized) && p.zmin;
        sMp[lp] = use_offset ? weight_offset<J>(vals + lp * LD, p.zmin[gp], p.flags) : 0.f;
    }
    fill_zero(acc, (int)Layout<J>::acc(npx, 5));
    __syncthreads();
    unsigned bad = 0;
    phase_resolve<J, true>(p, T, vals, sMp, acc, true, npx, bad);
    flush_bad(bad, p.err);
    __syncthreads();
    if (gp < 0) return;
    const float R = sum_copies(acc, npx, 0, lp), G = sum_copies(acc, npx, 1, lp);
    const float B = sum_copies(acc, npx, 2, lp), W = sum_copies(acc, npx, 3, lp);
    const float S = sum_copies(acc, npx, 4, lp);
    if (COMPOSITE) {
        composite_pixel(p, gp, R, G, B, W, S);
    } else {
        float *a = p.accum + 5 * gp;
        if (p.flags & kAccumulate) {
            a[0] += R;
            a[1] += G;
            a[2] += B;
            a[3] += W;
            a[4] += S;
        } else {
            a[0] = R;
            a[1] = G;
            a[2] = B;
            a[3] = W;
            a[4] = S;
        }
    }
}

// Steps 2-4 fused: coefficients never leave the SM between build and resolve.
template <int J, typename CT>
__global__ void __launch_bounds__(kThreads, MinBlocks<J>::value) k_fused(Params p) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD;
    extern __shared__ __align__(16) unsigned char smem[];
    const int npx = p.g.tile_w * p.g.tile_h;
    float *sF = reinterpret_cast<float *>(smem);
    float *sG = reinterpret_cast<float *>(smem + Layout<J>::plane(npx));
    float *vals = sF;  // the bin values replace the F bins after the barrier
    float *acc = sG;   // the accumulators replace the G bins
    float *sS = reinterpret_cast<float *>(smem + Layout<J>::region(npx));
    float *sMp = reinterpret_cast<float *>(smem + Layout<J>::region(npx) + Layout<J>::words(npx));
    unsigned *sZ =
        reinterpret_cast<unsigned *>(smem + Layout<J>::region(npx) + 2 * Layout<J>::words(npx));
    const Tile T = tile_of(p, blockIdx.x, true);
    fill_zero(smem, (int)(2 * Layout<J>::plane(npx)));
    for (int i = threadIdx.x; i < npx; i += blockDim.x) sZ[i] = 0x7f800000u;
    __syncthreads();
    unsigned bad = 0;
    phase_bins<J>(p, T, sF, sG, sZ, bad);
    flush_bad(bad, p.err);
    __syncthreads();
    const int lp = threadIdx.x;
    int64_t gp = -1;
    if (lp < npx) gp = global_pixel(p, T, lp);
    float v[C], S = 0.f;
    if (gp >= 0) {
        bins_to_coeffs<J>(sF + lp * LD, sG + lp * LD, v, S);
#pragma unroll
        for (int i = 0; i < C; ++i) v[i] = Cvt<CT>::from(Cvt<CT>::to(v[i]));  // storage precision
        if (p.coeff) store_row<CT, C>(static_cast<CT *>(p.coeff) + gp * C, v);
        if (p.zmin) p.zmin[gp] = __uint_as_float(sZ[lp]);
        coeffs_to_bins<J>(v);
#pragma unroll
        for (int i = 0; i < C; ++i) v[i] *= kLog2e;
    }
    __syncthreads();  // every bin row has been read
    if (gp >= 0) {
        put_vals<J>(vals + lp * LD, v);
        sS[lp] = S;
        sMp[lp] = (p.flags & kNormalized)
                      ? weight_offset<J>(vals + lp * LD, __uint_as_float(sZ[lp]), p.flags)
                      : 0.f;
    }
    fill_zero(acc, (int)Layout<J>::acc(npx, 4));
    __syncthreads();
    phase_resolve<J, false>(p, T, vals, sMp, acc, false, npx, bad);
    __syncthreads();
    if (gp < 0) return;
    composite_pixel(p, gp, sum_copies(acc, npx, 0, lp), sum_copies(acc, npx, 1, lp),
                    sum_copies(acc, npx, 2, lp), sum_copies(acc, npx, 3, lp), sS[lp]);
}

// Evaluation at arbitrary (pixel, depth) queries: J+1 coefficient reads per
// bin value, the same arithmetic as the tile kernels (in natural units).
template <int J, typename CT>
__global__ void __launch_bounds__(kThreads)
    k_absorbance(Params p, int64_t q, const uint32_t *__restrict__ qpx, const float *__restrict__ qz,
                 const float *__restrict__ qal, float *__restrict__ outA) {
    constexpr int C = Shape<J>::C;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= q) return;
    const uint32_t px = qpx[i];
    const float z = qz[i];
    const float al = qal ? qal[i] : 0.f;
    if ((int64_t)px >= (int64_t)p.g.width * p.g.height || !(z == z) || !(al == al)) {
        outA[i] = __int_as_float(0x7fc00000);
        atomicAdd(p.err, 1ull);
        return;
    }
    const CT *c = static_cast<const CT *>(p.coeff) + (int64_t)px * C;
    auto bin = [&](int m) {
        float A = Cvt<CT>::from(c[0]);
#pragma unroll
        for (int n = 0; n < J; ++n) {
            const float d = sqrt2_pow(n) * Cvt<CT>::from(c[(1 << n) + (m >> (J - n))]);
            A = ((m >> (J - 1 - n)) & 1) ? A - d : A + d;
        }
        return A;
    };
    const float s = clamp_depth(z) * (float)C;
    const int m = (int)s;
    const float f = s - (float)m;
    const float a = qal ? step_of(clamp_alpha(al)) : 0.f;
    float full, self;
    if (p.flags & kLinear) {
        const float pos = s - 0.5f;
        const int lo = min(max((int)floorf(pos), 0), C - 2);
        const float t = fminf(fmaxf(pos - (float)lo, 0.f), 1.f);
        const float A0 = bin(lo), A1 = bin(lo + 1);
        full = fmaf(t, A1 - A0, A0);
        const float B0 = lo < m ? 0.f : (lo == m ? 1.f - f : 1.f);
        const float B1 = lo + 1 < m ? 0.f : (lo + 1 == m ? 1.f - f : 1.f);
        self = a * fmaf(t, B1 - B0, B0);
    } else {
        full = bin(m);
        self = a * (1.f - f);
    }
    outA[i] = (qal && (p.flags & kSelfExclude)) ? fmaxf(full - self, 0.f) : full;
}

// ---------------------------------------------------------------- launchers

template <int J, typename CT> cudaError_t launch_build_t(const Params &p, int ntiles, cudaStream_t s) {
    const int npx = p.g.tile_w * p.g.tile_h;
    const size_t bytes = Layout<J>::build(npx);
    cudaError_t e = cudaFuncSetAttribute(k_build<J, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_build<J, CT><<<ntiles, kThreads, bytes, s>>>(p);
    return cudaGetLastError();
}

template <int J, typename CT, bool COMPOSITE>
cudaError_t launch_resolve_t(const Params &p, int ntiles, cudaStream_t s) {
    const int npx = p.g.tile_w * p.g.tile_h;
    const size_t bytes = Layout<J>::resolve(npx);
    cudaError_t e = cudaFuncSetAttribute(k_resolve<J, CT, COMPOSITE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_resolve<J, CT, COMPOSITE><<<ntiles, kThreads, bytes, s>>>(p);
    return cudaGetLastError();
}

template <int J, typename CT> cudaError_t launch_fused_t(const Params &p, int ntiles, cudaStream_t s) {
    const int npx = p.g.tile_w * p.g.tile_h;
    const size_t bytes = Layout<J>::fused(npx);
    cudaError_t e = cudaFuncSetAttribute(k_fused<J, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_fused<J, CT><<<ntiles, kThreads, bytes, s>>>(p);
    return cudaGetLastError();
}

template <int J, typename CT>
cudaError_t launch_absorbance_t(const Params &p, int64_t q, const uint32_t *qpx, const float *qz,
                                const float *qal, float *outA, cudaStream_t s) {
    if (q == 0) return cudaSuccess;
    const int64_t blocks = (q + kThreads - 1) / kThreads;
    k_absorbance<J, CT><<<(unsigned)blocks, kThreads, 0, s>>>(p, q, qpx, qz, qal, outA);
    return cudaGetLastError();
}

}  // namespace wt

// One translation unit per storage type instantiates every J.
#define WT_INSTANTIATE_TABLES(CT, IDX)                                                              \
    namespace wt {                                                                                 \
    const TileLaunch kBuild##IDX[5] = {launch_build_t<1, CT>, launch_build_t<2, CT>,               \
                                       launch_build_t<3, CT>, launch_build_t<4, CT>,               \
                                       launch_build_t<5, CT>};                                     \
    const TileLaunch kResolve##IDX[5] = {launch_resolve_t<1, CT, false>, launch_resolve_t<2, CT, false>, \
                                         launch_resolve_t<3, CT, false>, launch_resolve_t<4, CT, false>, \
                                         launch_resolve_t<5, CT, false>};                          \
    const TileLaunch kResolveComp##IDX[5] = {                                                      \
        launch_resolve_t<1, CT, true>, launch_resolve_t<2, CT, true>, launch_resolve_t<3, CT, true>, \
        launch_resolve_t<4, CT, true>, launch_resolve_t<5, CT, true>};                             \
    const TileLaunch kFused##IDX[5] = {launch_fused_t<1, CT>, launch_fused_t<2, CT>,               \
                                       launch_fused_t<3, CT>, launch_fused_t<4, CT>,               \
                                       launch_fused_t<5, CT>};                                     \
    const QueryLaunch kAbsorbance##IDX[5] = {                                                      \
        launch_absorbance_t<1, CT>, launch_absorbance_t<2, CT>, launch_absorbance_t<3, CT>,       \
        launch_absorbance_t<4, CT>, launch_absorbance_t<5, CT>};                                   \
    }
