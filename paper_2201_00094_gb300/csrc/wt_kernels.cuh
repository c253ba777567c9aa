// Kernels of the Wavelet OIT hot path.  One CTA per screen tile, 256 threads.
// Instantiated per J (1..5) and coefficient storage type in wt_kernels_*.cu.
#pragma once

#include "wt_internal.h"
#include "wt_tile.cuh"

namespace wt {

// Layout of the fused kernel: bin rows, then a second region that first holds
// the G bins and later the m_p + 5 accumulators, then the depth words.
template <int J> struct FusedSmem {
    static constexpr size_t second(int npx) {
        return (size_t)(npx * Shape<J>::LD > 6 * npx ? npx * Shape<J>::LD : 6 * npx);
    }
    static constexpr size_t total(int npx) { return (size_t)npx * Shape<J>::LD + second(npx) + npx; }
};

// §2.1 step 2: build the tile's coefficients and store them once.
template <int J, typename CT>
__global__ void __launch_bounds__(kThreads) k_build(Params p) {
    constexpr int LD = Shape<J>::LD;
    extern __shared__ float smem[];
    const int npx = p.g.tile_w * p.g.tile_h;
    float *sF = smem;
    float *sG = sF + npx * LD;
    unsigned *sZ = reinterpret_cast<unsigned *>(sG + npx * LD);
    const Tile T = tile_of(p, blockIdx.x, true);
    fill_smem(sF, 2 * npx * LD, 0.f);
    for (int i = threadIdx.x; i < npx; i += blockDim.x) sZ[i] = 0x7f800000u;  // +inf
    __syncthreads();
    unsigned bad = 0;
    phase_bins<J>(p, T, sF, sG, sZ, bad);
    flush_bad(bad, p.err);
    __syncthreads();
    phase_bins_to_coeffs<J>(sF, sG, npx);
    __syncthreads();
    const bool acc = (p.flags & kAccumulate) != 0;
    round_store_coeffs<J, CT>(p, T, sF, true, acc);
    if (p.zmin) store_zmin(p, T, sZ, npx, acc);
}

// §2.1 step 3 (+ step 4 when COMPOSITE): resolve against stored coefficients.
template <int J, typename CT, bool COMPOSITE>
__global__ void __launch_bounds__(kThreads) k_resolve(Params p) {
    constexpr int LD = Shape<J>::LD;
    extern __shared__ float smem[];
    const int npx = p.g.tile_w * p.g.tile_h;
    float *sA = smem;
    float *sMp = sA + npx * LD;
    float *sAcc = sMp + npx;
    const Tile T = tile_of(p, blockIdx.x, true);
    load_coeffs<J, CT>(p, T, sA);
    fill_smem(sAcc, 5 * npx, 0.f);
    __syncthreads();
    phase_coeffs_to_bins<J>(sA, npx);
    __syncthreads();
    const bool use_offset = (p.flags & kNormalized) && p.zmin;
    for (int lp = threadIdx.x; lp < npx; lp += blockDim.x) {
        const int64_t gp = global_pixel(p, T, lp);
        sMp[lp] = (use_offset && gp >= 0) ? weight_offset<J>(sA + lp * LD, p.zmin[gp], p.flags) : 0.f;
    }
    __syncthreads();
    unsigned bad = 0;
    phase_resolve<J, true>(p, T, sA, sMp, sAcc, npx, bad);
    flush_bad(bad, p.err);
    __syncthreads();
    resolve_epilogue<COMPOSITE>(p, T, sAcc, npx);
}

// Steps 2-4 fused: coefficients never leave the SM between build and resolve.
template <int J, typename CT>
__global__ void __launch_bounds__(kThreads) k_fused(Params p) {
    constexpr int LD = Shape<J>::LD;
    extern __shared__ float smem[];
    const int npx = p.g.tile_w * p.g.tile_h;
    float *sF = smem;
    float *sG = sF + npx * LD;
    unsigned *sZ = reinterpret_cast<unsigned *>(sG + FusedSmem<J>::second(npx));
    const Tile T = tile_of(p, blockIdx.x, true);
    fill_smem(sF, npx * LD + (int)FusedSmem<J>::second(npx), 0.f);
    for (int i = threadIdx.x; i < npx; i += blockDim.x) sZ[i] = 0x7f800000u;
    __syncthreads();
    unsigned bad = 0;
    phase_bins<J>(p, T, sF, sG, sZ, bad);
    flush_bad(bad, p.err);
    __syncthreads();
    phase_bins_to_coeffs<J>(sF, sG, npx);
    __syncthreads();
    round_store_coeffs<J, CT>(p, T, sF, p.coeff != nullptr, false);
    if (p.zmin) store_zmin(p, T, sZ, npx, false);
    float *sMp = sG;
    float *sAcc = sG + npx;
    fill_smem(sG, 6 * npx, 0.f);
    __syncthreads();
    phase_coeffs_to_bins<J>(sF, npx);
    __syncthreads();
    if (p.flags & kNormalized)
        for (int lp = threadIdx.x; lp < npx; lp += blockDim.x)
            sMp[lp] = weight_offset<J>(sF + lp * LD, __uint_as_float(sZ[lp]), p.flags);
    __syncthreads();
    phase_resolve<J, false>(p, T, sF, sMp, sAcc, npx, bad);
    __syncthreads();
    resolve_epilogue<true>(p, T, sAcc, npx);
}

// Evaluation at arbitrary (pixel, depth) queries: J+1 coefficient reads per bin.
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
            A += ((m >> (J - 1 - n)) & 1) ? -d : d;
        }
        return A;
    };
    const float zc = clamp_depth(z);
    const float s = zc * (float)C;
    const int m = (int)s;
    const float f = s - (float)m;
    const float a = qal ? step_of(clamp_alpha(al)) : 0.f;
    // bin values at m-1, m, m+1 (clamped); same arithmetic as the tile kernels
    float Abuf[3];
    Abuf[0] = bin(max(m - 1, 0));
    Abuf[1] = bin(m);
    Abuf[2] = bin(min(m + 1, C - 1));
    float self;
    float full;
    if (!(p.flags & kLinear)) {
        self = a * (1.f - f);
        full = Abuf[1];
    } else if (f < 0.5f) {
        if (m == 0) {
            self = a * (1.f - f);
            full = Abuf[1];
        } else {
            const float t = f + 0.5f;
            self = a * (1.f - f) * t;
            full = fmaf(t, Abuf[1] - Abuf[0], Abuf[0]);
        }
    } else if (m == C - 1) {
        self = a * (1.f - f);
        full = Abuf[1];
    } else {
        const float t = f - 0.5f;
        self = a * fmaf(1.f - f, 1.f - t, t);
        full = fmaf(t, Abuf[2] - Abuf[1], Abuf[1]);
    }
    outA[i] = (qal && (p.flags & kSelfExclude)) ? fmaxf(full - self, 0.f) : full;
}

// ---------------------------------------------------------------- launchers

template <int J, typename CT> cudaError_t launch_build_t(const Params &p, int ntiles, cudaStream_t s) {
    const int npx = p.g.tile_w * p.g.tile_h;
    const size_t bytes = Smem<J>::bins(npx) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_build<J, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_build<J, CT><<<ntiles, kThreads, bytes, s>>>(p);
    return cudaGetLastError();
}

template <int J, typename CT, bool COMPOSITE>
cudaError_t launch_resolve_t(const Params &p, int ntiles, cudaStream_t s) {
    const int npx = p.g.tile_w * p.g.tile_h;
    const size_t bytes = Smem<J>::resolve(npx) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_resolve<J, CT, COMPOSITE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_resolve<J, CT, COMPOSITE><<<ntiles, kThreads, bytes, s>>>(p);
    return cudaGetLastError();
}

template <int J, typename CT> cudaError_t launch_fused_t(const Params &p, int ntiles, cudaStream_t s) {
    const int npx = p.g.tile_w * p.g.tile_h;
    const size_t bytes = FusedSmem<J>::total(npx) * sizeof(float);
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
