// Kernels of the Wavelet OIT hot path.  One CTA per screen tile, 256 threads.
// Instantiated per J (1..5) and coefficient storage type in wt_kernels_*.cu.
#pragma once

#include "wt_internal.h"
#include "wt_tile.cuh"

namespace wt {

// Blocks per SM the kernels are compiled for (caps registers per thread so
// that shared memory, not registers, sets the occupancy).
template <int J> struct MinBlocks { static constexpr int value = J >= 6 ? 1 : (J == 5 ? 3 : 4); };
// Tiles of at most this many pixels fit four fused blocks per SM at J = 5.
constexpr int kFourBlockTilePx = 192;

// §2.1 step 2: build the tile's coefficients and store them once.
template <int J, typename CT, int MB = MinBlocks<J>::value>
__global__ void __launch_bounds__(kThreads, MB) k_build(Params p) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD;
    extern __shared__ __align__(16) unsigned char smem[];
    const int npx = p.g.tile_w * p.g.tile_h;
    unsigned *sF = reinterpret_cast<unsigned *>(smem);
    unsigned *sG = reinterpret_cast<unsigned *>(smem + Layout<J>::plane(npx));
    unsigned *sZ = reinterpret_cast<unsigned *>(smem + 2 * Layout<J>::plane(npx));
    const Tile T = tile_of(p, blockIdx.x, true);
    prefetch_tile<kWithZ>(p, T);
    fill_zero(smem, (int)(2 * Layout<J>::plane(npx)));
    for (int i = threadIdx.x; i < npx; i += blockDim.x) sZ[i] = 0x7f800000u;  // +inf
    __syncthreads();
    unsigned bad = 0;
    const bool scaled = phase_bins<J>(p, T, sF, sG, sZ, bad);
    flush_bad(bad, p.err);
    const int lp = threadIdx.x;
    int64_t gp = -1;
    if (lp < npx) gp = global_pixel(p, T, lp);
    CT *coeff = static_cast<CT *>(p.coeff);
    const bool acc = (p.flags & kAccumulate) != 0;
    // rows of whole 16-byte chunks go out through a staging copy over the F
    // bins (coalesced stores); accumulation adds to the stored rows directly
    const bool stage = Staged<CT, C>::ok && !acc;
    const int64_t P = (int64_t)p.g.width * p.g.height;
    float c[C], S;
    int e = 0;  // the row's shared exponent (WT_SE16)
    if (gp >= 0) {
        bins_to_coeffs<J>(sF + lp * LD, sG + lp * LD, c, S, scaled);
        CT *dst = coeff + gp * C;
        if (acc) {
            float old[C];
            load_row<CT, C>(dst, old, kIsSE16<CT> ? (int)se16_expo<C>(coeff, P)[gp] - kSE16Bias : 0);
#pragma unroll
            for (int i = 0; i < C; ++i) c[i] += old[i];
        }
        e = storage_exponent<CT, C>(c);
        if constexpr (kIsSE16<CT>) se16_expo<C>(coeff, P)[gp] = (uint8_t)(e + kSE16Bias);
        if (!stage) store_row<CT, C>(dst, c, e);
        if (p.zmin) {
            float v = __uint_as_float(sZ[lp]);
            if (acc) v = fminf(v, p.zmin[gp]);
            p.zmin[gp] = v;
        }
        if (p.total) p.total[gp] = acc ? p.total[gp] + S : S;
    }
    if (stage) {
        uint4 *st = reinterpret_cast<uint4 *>(smem);
        __syncthreads();  // every bin row has been read
        if (gp >= 0) stage_row<CT, C>(st, lp, c, e);
        __syncthreads();
        copy_staged<CT, C>(p, T, st, npx * Staged<CT, C>::K * 16, coeff);
    }
}

// §2.1 step 3 (+ step 4 when COMPOSITE): resolve against stored coefficients.
// DEF and MB as for k_fused: DEF when the reading flags (accumulation aside)
// are the default, MB the blocks per SM the registers are budgeted for.
template <int J, typename CT, bool COMPOSITE, bool DEF = false, int MB = MinBlocks<J>::value>
__global__ void __launch_bounds__(kThreads, MB) k_resolve(Params p) {
    constexpr int C = Shape<J>::C, LDV = Shape<J>::LDV;
    extern __shared__ __align__(16) unsigned char smem[];
    const int npx = p.g.tile_w * p.g.tile_h;
    float *vals = reinterpret_cast<float *>(smem);
    float4 *accw = reinterpret_cast<float4 *>(smem + Layout<J>::vplane(npx));
    float *sS = reinterpret_cast<float *>(smem + Layout<J>::vplane(npx) + Layout<J>::accw(npx));
    const Tile T = tile_of(p, blockIdx.x, true);
    prefetch_tile<kWithZ | kWithRGB>(p, T);
    const int lp = threadIdx.x;
    int64_t gp = -1;
    if (lp < npx) gp = global_pixel(p, T, lp);
    // rows of whole 16-byte chunks come in through a staging copy over the
    // (not yet used) accumulator area (coalesced loads)
    const CT *coeff = static_cast<const CT *>(p.coeff);
    uint4 *st = reinterpret_cast<uint4 *>(accw);
    if (Staged<CT, C>::ok) {
        load_staged<CT, C>(p, T, st, coeff);
        __syncthreads();
    }
    if (gp >= 0) {
        float v[C];
        const int e = kIsSE16<CT> ? (int)se16_expo<C>(coeff, (int64_t)p.g.width * p.g.height)[gp] - kSE16Bias : 0;
        if (Staged<CT, C>::ok) unstage_row<CT, C>(st, lp, v, e);
        else load_row<CT, C>(coeff + gp * C, v, e);
        coeffs_to_bins<J>(v, kLog2e);
        put_bins<J>(vals + lp * LDV, v, p.zmin ? p.zmin[gp] : __int_as_float(0x7f800000),
                    DEF ? kDefaultFlags : p.flags);
    }
    if (Staged<CT, C>::ok) __syncthreads();  // staged rows consumed
    fill_zero(accw, (int)(Layout<J>::accw(npx) + Layout<J>::words(npx)));
    __syncthreads();
    unsigned bad = 0;
    // with the build's totals the steps need not be summed again (and the own
    // step of the self-exclusion comes from the hardware log2, as in the
    // fused kernel)
    phase_resolve<J, true, DEF>(p, T, vals, accw, p.total ? nullptr : sS, bad);
    flush_bad(bad, p.err);
    __syncthreads();
    if (gp < 0) return;
    const float4 a = sum_warps(accw, npx, lp);
    const float S = p.total ? p.total[gp] : sS[lp];
    if (COMPOSITE) {
        composite_pixel(p, gp, a.x, a.y, a.z, a.w, S);
    } else {
        float *o = p.accum + 5 * gp;
        if (p.flags & kAccumulate) {
            o[0] += a.x;
            o[1] += a.y;
            o[2] += a.z;
            o[3] += a.w;
            o[4] += S;
        } else {
            o[0] = a.x;
            o[1] = a.y;
            o[2] = a.z;
            o[3] = a.w;
            o[4] = S;
        }
    }
}

// Steps 2-4 fused for one tile: the coefficients never leave the SM between
// build and resolve.  Ends with a barrier, so a persistent caller may reuse the
// shared memory for its next tile.
template <int J, typename CT, bool DEF = false>
__device__ __forceinline__ void fused_tile(const Params &p, int tile, unsigned char *smem) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD, LDV = Shape<J>::LDV;
    const int npx = p.g.tile_w * p.g.tile_h;
    unsigned *sF = reinterpret_cast<unsigned *>(smem);
    unsigned *sG = reinterpret_cast<unsigned *>(smem + Layout<J>::plane(npx));
    // after the build: bin values over the F bins, then the warps'
    // accumulators and the S words over the G bins
    float *vals = reinterpret_cast<float *>(smem);
    float4 *accw = reinterpret_cast<float4 *>(smem + Layout<J>::vplane(npx));
    float *sS = reinterpret_cast<float *>(smem + Layout<J>::vplane(npx) + Layout<J>::accw(npx));
    unsigned *sZ = reinterpret_cast<unsigned *>(smem + Layout<J>::region(npx));
    const Tile T = tile_of(p, tile, true);
    prefetch_tile<kWithZ | kWithRGB>(p, T);
    fill_zero(smem, (int)(2 * Layout<J>::plane(npx)));
    for (int i = threadIdx.x; i < npx; i += blockDim.x) sZ[i] = 0x7f800000u;
    __syncthreads();
    unsigned bad = 0;
    const bool scaled = phase_bins<J>(p, T, sF, sG, sZ, bad);
    flush_bad(bad, p.err);
    const int lp = threadIdx.x;
    int64_t gp = -1;
    if (lp < npx) gp = global_pixel(p, T, lp);
    // the coefficient rows go out through a staging copy over the (not yet
    // used) accumulator area when they are whole 16-byte chunks
    CT *coeff = static_cast<CT *>(p.coeff);
    const bool stage = Staged<CT, C>::ok && coeff != nullptr;
    float v[C], S = 0.f;
    int e = 0;  // the row's shared exponent (WT_SE16)
    if (gp >= 0) {
        bins_to_coeffs<J>(sF + lp * LD, sG + lp * LD, v, S, scaled);
        e = round_row<CT, C>(v);  // storage precision: the resolve uses the stored values
        if constexpr (kIsSE16<CT>) {
            if (coeff) se16_expo<C>(coeff, (int64_t)p.g.width * p.g.height)[gp] = (uint8_t)(e + kSE16Bias);
        }
        if (coeff && !stage) store_row<CT, C>(coeff + gp * C, v, e);
        if (p.zmin) p.zmin[gp] = __uint_as_float(sZ[lp]);
    }
    __syncthreads();  // every bin row has been read
    if (gp >= 0) {
        if (stage) stage_row<CT, C>(reinterpret_cast<uint4 *>(accw), lp, v, e);
        coeffs_to_bins<J>(v, kLog2e);
        put_bins<J>(vals + lp * LDV, v, __uint_as_float(sZ[lp]), DEF ? kDefaultFlags : p.flags);
        sS[lp] = S;
    }
    if (stage) {
        __syncthreads();  // staged rows complete
        copy_staged<CT, C>(p, T, reinterpret_cast<uint4 *>(accw), (int)Layout<J>::accw(npx), coeff);
    } else {
        fill_zero(accw, (int)Layout<J>::accw(npx));
    }
    __syncthreads();
    phase_resolve<J, false, DEF>(p, T, vals, accw, nullptr, bad);
    __syncthreads();
    if (gp >= 0) {
        const float4 a = sum_warps(accw, npx, lp);
        composite_pixel(p, gp, a.x, a.y, a.z, a.w, sS[lp]);
        if (p.accum) {  // the pixel sums, for the adjoint
            float *o = p.accum + 5 * gp;
            o[0] = a.x;
            o[1] = a.y;
            o[2] = a.z;
            o[3] = a.w;
            o[4] = sS[lp];
        }
    }
    __syncthreads();
}

// DEF: compiled for the default flags (p.flags == kDefaultFlags), so the
// per-fragment reconstruction carries no flag tests.  MB: blocks per SM the
// registers are budgeted for; at J = 5 a tile of at most 192 pixels leaves
// room for four blocks' shared memory, so that launch caps registers at 64.
template <int J, typename CT, bool DEF, int MB>
__global__ void __launch_bounds__(kThreads, MB) k_fused(Params p) {
    extern __shared__ __align__(16) unsigned char smem[];
    fused_tile<J, CT, DEF>(p, p.tile0 + (int)blockIdx.x, smem);
}

// The single-pass variant the paper proposes (§4): every fragment of frame t
// is resolved against frame t-1's coefficients, which are complete before the
// frame starts, and frame t's coefficients are built for the next frame; no
// pass waits for the build.  With a static scene the result equals the
// two-pass method's; with motion it is the paper's approximation (visibility
// from the previous frame).  The weight offset comes from frame t-1's near
// bound; exponents are clamped to [0, 120] so that fragments nearer or much
// farther than anything in frame t-1 keep finite, non-zero weights.
// Within a tile, the resolve against frame t-1 (its bin values and the
// warps' accumulators) comes first and the build of frame t (F and G bins)
// second, over the tile's own fragment range both times: each fragment comes
// from HBM once (the second read hits L2), and the two phases share the fused
// kernel's shared-memory region.
template <int J> struct TemporalLayout {
    static constexpr size_t total(int npx) { return Layout<J>::fused(npx); }
};

template <int J, typename CT, bool DEF, int MB>
__global__ void __launch_bounds__(kThreads, MB) k_temporal(Params p, const void *coeff_prev, const float *zmin_prev) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD, LDV = Shape<J>::LDV;
    extern __shared__ __align__(16) unsigned char smem[];
    const int npx = p.g.tile_w * p.g.tile_h;
    float *vals = reinterpret_cast<float *>(smem);
    float4 *accw = reinterpret_cast<float4 *>(smem + Layout<J>::vplane(npx));
    unsigned *sF = reinterpret_cast<unsigned *>(smem);
    unsigned *sG = reinterpret_cast<unsigned *>(smem + Layout<J>::plane(npx));
    unsigned *sZ = reinterpret_cast<unsigned *>(smem + Layout<J>::region(npx));
    uint4 *st = reinterpret_cast<uint4 *>(accw);  // staging of coefficient rows
    const uint32_t flags = DEF ? kDefaultFlags : p.flags;
    const Tile T = tile_of(p, p.tile0 + (int)blockIdx.x, true);
    prefetch_tile<kWithZ | kWithRGB>(p, T);
    const int lp = threadIdx.x;
    int64_t gp = -1;
    if (lp < npx) gp = global_pixel(p, T, lp);
    const int64_t P = (int64_t)p.g.width * p.g.height;
    // frame t-1's coefficients -> bin values (log2 units, its weight offset folded in)
    const CT *prev = static_cast<const CT *>(coeff_prev);
    if (Staged<CT, C>::ok) {
        load_staged<CT, C>(p, T, st, prev);
        __syncthreads();
    }
    if (gp >= 0) {
        float v[C];
        const int e = kIsSE16<CT> ? (int)se16_expo<C>(prev, P)[gp] - kSE16Bias : 0;
        if (Staged<CT, C>::ok) unstage_row<CT, C>(st, lp, v, e);
        else load_row<CT, C>(prev + gp * C, v, e);
        coeffs_to_bins<J>(v, kLog2e);
        put_bins<J>(vals + lp * LDV, v, zmin_prev ? zmin_prev[gp] : __int_as_float(0x7f800000), flags);
    }
    __syncthreads();  // staged rows consumed
    fill_zero(accw, (int)Layout<J>::accw(npx));
    __syncthreads();
    // the resolve of frame t's fragments against frame t-1's visibility
    unsigned bad = 0;
    phase_resolve<J, false, DEF, true>(p, T, vals, accw, nullptr, bad);
    __syncthreads();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gp >= 0) acc = sum_warps(accw, npx, lp);
    __syncthreads();  // bin values and accumulators consumed: the region takes frame t's bins
    fill_zero(smem, (int)(2 * Layout<J>::plane(npx)));
    for (int i = threadIdx.x; i < npx; i += blockDim.x) sZ[i] = 0x7f800000u;
    __syncthreads();
    // frame t's build (fixed-scale bins, per-pixel scales as the fallback)
    const bool scaled = phase_bins<J>(p, T, sF, sG, sZ, bad);
    flush_bad(bad, p.err);
    float c[C], S = 0.f;
    if (gp >= 0) bins_to_coeffs<J>(sF + lp * LD, sG + lp * LD, c, S, scaled);
    __syncthreads();  // every bin row read: the region stages the new coefficients
    CT *next = static_cast<CT *>(p.coeff);
    const bool stage = Staged<CT, C>::ok && next != nullptr;
    if (gp >= 0) {
        composite_pixel(p, gp, acc.x, acc.y, acc.z, acc.w, S);
        if (p.zmin) p.zmin[gp] = __uint_as_float(sZ[lp]);
        if (next) {
            const int e = storage_exponent<CT, C>(c);
            if constexpr (kIsSE16<CT>) se16_expo<C>(next, P)[gp] = (uint8_t)(e + kSE16Bias);
            if (stage) stage_row<CT, C>(st, lp, c, e);
            else store_row<CT, C>(next + gp * C, c, e);
        }
    }
    if (stage) {
        __syncthreads();
        copy_staged<CT, C>(p, T, st, npx * Staged<CT, C>::K * 16, next);
    }
}

template <int J, typename CT, bool DEF, int MB>
cudaError_t launch_temporal_k(const Params &p, int ntiles, const void *coeff_prev, const float *zmin_prev,
                              cudaStream_t s) {
    const int npx = p.g.tile_w * p.g.tile_h;
    const size_t bytes = TemporalLayout<J>::total(npx);
    if (bytes > kMaxSmemPerBlock) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(k_temporal<J, CT, DEF, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bytes);
    if (e != cudaSuccess) return e;
    k_temporal<J, CT, DEF, MB><<<ntiles, kThreads, bytes, s>>>(p, coeff_prev, zmin_prev);
    return cudaGetLastError();
}
template <int J, typename CT>
cudaError_t launch_temporal_t(const Params &p, int ntiles, const void *coeff_prev, const float *zmin_prev,
                              cudaStream_t s) {
    // the fused kernel's shared memory and register budgets
    const bool def = p.flags == kDefaultFlags;
    if constexpr (J == 5) {
        if (p.g.tile_w * p.g.tile_h <= kFourBlockTilePx)
            return def ? launch_temporal_k<J, CT, true, 4>(p, ntiles, coeff_prev, zmin_prev, s)
                       : launch_temporal_k<J, CT, false, 4>(p, ntiles, coeff_prev, zmin_prev, s);
    }
    return def ? launch_temporal_k<J, CT, true, MinBlocks<J>::value>(p, ntiles, coeff_prev, zmin_prev, s)
               : launch_temporal_k<J, CT, false, MinBlocks<J>::value>(p, ntiles, coeff_prev, zmin_prev, s);
}

// Serving: one persistent launch works through the tile tasks of several
// frames (continuous batching).  The step's task table lists, per admitted
// frame, a slot and a range of its tiles; tasks are numbered by the running
// sum of the range lengths, and CTAs claim task numbers from a device counter.
template <int J, typename CT>
__global__ void __launch_bounds__(kThreads, MinBlocks<J>::value)
    k_serve(const Params *__restrict__ slots, const ServeTask *__restrict__ tasks, int ntasks,
            int64_t total, unsigned long long *counter) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long claim;
    for (;;) {
        if (threadIdx.x == 0) claim = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long k = claim;
        __syncthreads();
        if (k >= total) return;
        int lo = 0, hi = ntasks - 1;  // last range with start <= k
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tasks[mid].start <= k) lo = mid;
            else hi = mid - 1;
        }
        const ServeTask t = tasks[lo];
        fused_tile<J, CT>(slots[t.slot], t.tile0 + (int)(k - t.start), smem);
    }
}

// ---------------------------------------------------------------- adjoint

// Shared-memory layout of the adjoint: F, G bins; later the bin values, the
// warps' accumulators and then the scattered adjoint bins Gamma; then ten
// per-pixel words (depth, S, u[3], ybar[3], const, Gamma's fixed-point scale).
template <int J> struct BackLayout {
    static constexpr size_t P(int npx) { return Layout<J>::plane(npx); }
    static constexpr size_t V(int npx) { return Layout<J>::vplane(npx); }
    static constexpr size_t W(int npx) { return Layout<J>::words(npx); }
    static constexpr size_t second(int npx) {
        return Layout<J>::accw(npx) > P(npx) ? Layout<J>::accw(npx) : P(npx);
    }
    static constexpr size_t region(int npx) {
        return 2 * P(npx) > V(npx) + second(npx) ? 2 * P(npx) : V(npx) + second(npx);
    }
    static constexpr size_t total(int npx) { return region(npx) + 10 * W(npx); }
};

// Re-derives everything the adjoint needs about one fragment from its inputs
// and the pixel's bin values (log2 units, shifted by m_p): local pixel (or -1),
// clamped alpha, position q, and weight w = alpha 2^-A'.  The own step
// removed under self-exclusion is -log2(1 - alpha) from the hardware log2, as
// in the forward sums the adjoint recomputes (phase_resolve without S).
template <int J> struct FragState {
    int lp;
    float ac, w;
    Pos q;
};
template <int J>
__device__ __forceinline__ FragState<J> frag_state(const Params &p, const Tile &T, const float *vals,
                                                   uint32_t px, float z, float al) {
    FragState<J> st;
    st.lp = -1;
    if (!(z == z) || !(al == al)) return st;
    st.lp = local_pixel(px, p, T);
    if (st.lp < 0) return st;
    st.ac = clamp_alpha(al);
    st.q = locate<J>(clamp_depth(z) * (float)(1 << J), p.flags);
    const float full = recon_at<J>(vals + st.lp * Shape<J>::LDV, st.q, p.flags);
    const float Ah = (p.flags & kSelfExclude) ? fmaxf(fmaf(lg2(1.f - st.ac), st.q.g, full), 0.f) : full;
    st.w = st.ac * ex2(-Ah);
    return st;
}

// Adjoint of build + resolve + composite (no counterpart in the paper; it
// follows from the linearity of the closed-form coefficients of §2.3.1).
// With g = dL/d(out) per pixel: u = g_rgb (1-T)/W and ybar = R/W (normalised;
// u = g_rgb, ybar = 0 literal), tau = g_rgb.(bg - ybar) - g_a.  Per fragment
// beta = u.(c - ybar), gamma = dL/dA = -beta w, dL/dc = u w.  Since
// A_i = sum_j a_j K(z_i, z_j) with K the reconstruction at z_i of a unit step
// at z_j, dL/da_j = sum_i gamma_i K(z_i, z_j) - T tau, and the sum is
// sum_m Gamma_m B^(j)_m with Gamma the gammas scattered into the bins with the
// interpolation weights and B^(j) the unit step's bin values (0, 1-f, 1):
// with the inclusive suffix Q_m = sum_{m'>=m} Gamma_m', it is
// (1 - f_j) Q_{m_j} + f_j Q_{m_j+1}; self-exclusion removes gamma_j g_j.
// dL/dalpha = beta 2^-A' + (dL/da) / (1 - alpha) inside the clamp, else 0.
// Coefficients are rebuilt here (never stored between the passes).
template <int J, typename CT, int MB>
__global__ void __launch_bounds__(kThreads, MB) k_backward(Params p) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD, LDV = Shape<J>::LDV;
    extern __shared__ __align__(16) unsigned char smem[];
    const int npx = p.g.tile_w * p.g.tile_h;
    const size_t PL = Layout<J>::plane(npx), VL = Layout<J>::vplane(npx), WD = Layout<J>::words(npx);
    unsigned *sF = reinterpret_cast<unsigned *>(smem);
    unsigned *sG = reinterpret_cast<unsigned *>(smem + PL);
    float *vals = reinterpret_cast<float *>(smem);
    float4 *accw = reinterpret_cast<float4 *>(smem + VL);
    float *gam = reinterpret_cast<float *>(smem + VL);  // replaces the accumulators
    unsigned char *wbase = smem + BackLayout<J>::region(npx);
    unsigned *sZ = reinterpret_cast<unsigned *>(wbase);
    float *sS = reinterpret_cast<float *>(wbase + WD);
    float *sU = reinterpret_cast<float *>(wbase + 2 * WD);  // 3 planes
    float *sY = reinterpret_cast<float *>(wbase + 5 * WD);  // 3 planes
    float *sK = reinterpret_cast<float *>(wbase + 8 * WD);
    float *sX = reinterpret_cast<float *>(wbase + 9 * WD);  // Gamma's scale 2^(30 - e) per pixel
    int *gi = reinterpret_cast<int *>(gam);                  // Gamma in fixed point
    const int wpl = (int)(WD / 4);  // floats per word plane
    const Tile T = tile_of(p, blockIdx.x, true);
    fill_zero(smem, (int)(2 * PL));
    for (int i = threadIdx.x; i < npx; i += blockDim.x) sZ[i] = 0x7f800000u;
    __syncthreads();
    unsigned bad = 0;
    const bool scaled = phase_bins<J>(p, T, sF, sG, sZ, bad);
    flush_bad(bad, p.err);
    const int lp = threadIdx.x;
    int64_t gp = -1;
    if (lp < npx) gp = global_pixel(p, T, lp);
    float v[C], S = 0.f;
    if (gp >= 0) {
        bins_to_coeffs<J>(sF + lp * LD, sG + lp * LD, v, S, scaled);
        round_row<CT, C>(v);  // the forward pass resolves with the stored values
        coeffs_to_bins<J>(v, kLog2e);
    }
    __syncthreads();
    if (gp >= 0) {
        put_bins<J>(vals + lp * LDV, v, __uint_as_float(sZ[lp]), p.flags);
        sS[lp] = S;
    }
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (p.accum) {  // the forward call's sums
        __syncthreads();
        if (gp >= 0) {
            const float *a = p.accum + 5 * gp;
            acc = make_float4(a[0], a[1], a[2], a[3]);
        }
    } else {  // the forward sums, recomputed
        fill_zero(accw, (int)Layout<J>::accw(npx));
        __syncthreads();
        phase_resolve<J, false>(p, T, vals, accw, nullptr, bad);
        __syncthreads();
        if (gp >= 0) acc = sum_warps(accw, npx, lp);
        __syncthreads();  // accumulators consumed; their space becomes Gamma
    }
    if (gp >= 0) {
        const float Tt = expf(-S), cover = -expm1f(-S);
        const float *go = p.gout + 4 * gp;
        float bgc[3] = {p.bg0, p.bg1, p.bg2};
        if (p.bg_img) {
            bgc[0] = p.bg_img[3 * gp];
            bgc[1] = p.bg_img[3 * gp + 1];
            bgc[2] = p.bg_img[3 * gp + 2];
        }
        const float Rc[3] = {acc.x, acc.y, acc.z};
        float tau = -go[3];
        for (int ch = 0; ch < 3; ++ch) {
            float u = 0.f, y = 0.f;
            if (p.flags & kNormalized) {
                if (acc.w > 0.f) {
                    u = go[ch] * cover / acc.w;
                    y = Rc[ch] / acc.w;
                    tau += go[ch] * (bgc[ch] - y);
                }
            } else {
                u = go[ch];
                tau += go[ch] * bgc[ch];
            }
            sU[ch * wpl + lp] = u;
            sY[ch * wpl + lp] = y;
        }
        sK[lp] = -Tt * tau;
        // sum |gamma| over the pixel <= (|u_r| + |u_g| + |u_b|) W when colours
        // lie in [0, 1]: the scale 2^(30 - e), B < 2^e, keeps that sum below
        // 2^30 (B is W up to FP32 rounding, and 2^e > B leaves a factor of up
        // to two).  A non-finite B comes with non-finite gammas, which pass 3
        // sends down the FP32 path.
        const float B = (fabsf(sU[lp]) + fabsf(sU[wpl + lp]) + fabsf(sU[2 * wpl + lp])) * acc.w;
        const int e = B > 0.f && B < 3.0e38f ? min(max(ilogbf(B) + 1, -90), 97) : 0;
        sX[lp] = exp2i(30 - e);
    }
    fill_zero(gam, (int)PL);
    __syncthreads();
    const uint32_t flags = p.flags;
    // pass 3: colour gradients and the scatter of gamma into the bins; each
    // fragment's gamma waits in its grad_alpha entry for pass 4 (read back by
    // the thread that wrote it: both passes split the range the same way).
    // The scatter adds rint(gamma s_p) with 32-bit integer atomics (order-free,
    // so the gradients are the same on every run).  The scale keeps a pixel's
    // sum of |gamma| s_p below 2^30 whenever its colours lie in [0, 1] (their
    // weighted mean then does too, and |beta| <= |u_r| + |u_g| + |u_b|), so no
    // word can wrap; a fragment with a colour outside [0, 1] (or NaN) sends
    // the tile through the pass again with FP32 atomics.
    auto pass3 = [&](auto fixed_tag) {
        constexpr bool FIXED = decltype(fixed_tag)::value;
        bool ovf = false;
        for_each_group<kWithZ | kWithRGB>(T.s, T.e, p, [&](auto &G) {
            constexpr int N = std::remove_reference_t<decltype(G)>::size;
            float gr[3][N], gm[N];
#pragma unroll
            for (int k = 0; k < N; ++k) {
                gr[0][k] = gr[1][k] = gr[2][k] = 0.f;
                gm[k] = 0.f;
                if (!G.v) continue;
                const FragState<J> st = frag_state<J>(p, T, vals, G.px[k], G.z[k], G.al[k]);
                if (st.lp < 0) continue;
                const float c[3] = {G.r[k], G.g[k], G.b[k]};
                float beta = 0.f;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    const float u = sU[ch * wpl + st.lp];
                    beta = fmaf(u, c[ch] - sY[ch * wpl + st.lp], beta);
                    gr[ch][k] = u * st.w;
                }
                const float gamma = -beta * st.w;
                gm[k] = gamma;
                if constexpr (FIXED)
                    ovf |= !(fminf(fminf(c[0], c[1]), c[2]) >= 0.f && fmaxf(fmaxf(c[0], c[1]), c[2]) <= 1.f &&
                             fabsf(gamma) <= 3.0e38f);
                const float sc = FIXED ? sX[st.lp] : 1.f;
                auto add = [&](int m, float x) {
                    if constexpr (FIXED) atomicAdd(&gi[st.lp * LD + m], __float2int_rn(x * sc));
                    else atomicAdd(&gam[st.lp * LD + m], x);
                };
                if (flags & kLinear) {
                    add(st.q.lo, gamma * (1.f - st.q.t));
                    add(st.q.lo + 1, gamma * st.q.t);
                } else {
                    add(st.q.m, gamma);
                }
            }
            if (G.v) {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) store_group<N>(p.grgb + ch * p.n, G.i0, gr[ch]);
                store_group<N>(p.galpha, G.i0, gm);
            }
        });
        return ovf;
    };
    const bool fp32 = __syncthreads_or(pass3(std::true_type{}));
    if (fp32) {  // rare: the tile again, in FP32 (its outputs are rewritten with the same values)
        fill_zero(gam, (int)PL);
        __syncthreads();
        pass3(std::false_type{});
    }
    __syncthreads();
    if (gp >= 0) {  // inclusive suffix sums Q_m, with Q_C = 0
        float *row = gam + lp * LD;
        row[C] = 0.f;
        if (!fp32) {  // exact integer sums, one rounding each
            const int *qi = gi + lp * LD;
            const float inv = 1.f / sX[lp];  // a power of two
            long long acc_q = 0;
            for (int m = C - 1; m >= 0; --m) {
                acc_q += qi[m];
                row[m] = (float)acc_q * inv;
            }
        } else {
            float acc_s = 0.f;
            for (int m = C - 1; m >= 0; --m) {
                acc_s += row[m];
                row[m] = acc_s;
            }
        }
    }
    __syncthreads();
    // pass 4: opacity gradients from each fragment's gamma (pass 3), its
    // position in its bin and the suffix sums:
    // dL/dalpha = beta 2^-A' + (dL/da) / (1 - alpha), beta 2^-A' = -gamma / alpha
    for_each_group<kWithZ>(T.s, T.e, p, [&](auto &G) {
        constexpr int N = std::remove_reference_t<decltype(G)>::size;
        float gm[N], ga[N];
        load_group<N>(p.galpha, G.i0, G.v, gm);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            ga[k] = 0.f;
            if (!G.v) continue;
            const float al = G.al[k];
            if (!(G.z[k] == G.z[k]) || !(al == al)) continue;
            const int lp = local_pixel(G.px[k], p, T);
            if (lp < 0) continue;
            const Pos q = locate<J>(clamp_depth(G.z[k]) * (float)(1 << J), flags);
            const float gamma = gm[k];
            const float *Q = gam + lp * LD;
            float da = fmaf(q.f, Q[q.m + 1], (1.f - q.f) * Q[q.m]);
            if (flags & kSelfExclude) da -= gamma * q.g;
            da += sK[lp];
            if (al > 0.f && al < kAlphaMax) ga[k] = da / (1.f - al) - gamma / al;
        }
        if (G.v) store_group<N>(p.galpha, G.i0, ga);
    });
}

template <int J, typename CT>
cudaError_t launch_serve_t(const Params *slots, const ServeTask *tasks, int ntasks, int64_t total,
                           unsigned long long *counter, int npx, int grid, cudaStream_t s) {
    const size_t bytes = Layout<J>::fused(npx);
    if (bytes > kMaxSmemPerBlock) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(k_serve<J, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_serve<J, CT><<<grid, kThreads, bytes, s>>>(slots, tasks, ntasks, total, counter);
    return cudaGetLastError();
}

// CTAs of a fused-tile kernel that fit on one SM (persistent grid sizing).
template <int J, typename CT> int serve_blocks_per_sm(int npx) {
    int n = 0;
    const size_t bytes = Layout<J>::fused(npx);
    if (bytes > kMaxSmemPerBlock) return 0;
    if (cudaFuncSetAttribute(k_serve<J, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_serve<J, CT>, kThreads, bytes) != cudaSuccess) return 0;
    return n;
}

template <int J, typename CT, int MB> cudaError_t launch_backward_k(const Params &p, int ntiles, cudaStream_t s) {
    const size_t bytes = BackLayout<J>::total(p.g.tile_w * p.g.tile_h);
    cudaError_t e =
        cudaFuncSetAttribute(k_backward<J, CT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_backward<J, CT, MB><<<ntiles, kThreads, bytes, s>>>(p);
    return cudaGetLastError();
}
// Registers budgeted for the CTAs per SM that the shared memory allows (228 KB
// per SM, 1 KB of it reserved per CTA): three when at least three fit (80
// registers, no spills), else two.  Four (64 registers) spill and were slower.
template <int J, typename CT> cudaError_t launch_backward_t(const Params &p, int ntiles, cudaStream_t s) {
    const size_t bytes = BackLayout<J>::total(p.g.tile_w * p.g.tile_h);
    if (bytes > kMaxSmemPerBlock) return cudaErrorNotSupported;
    if (3 * (bytes + 1024) <= 233472) return launch_backward_k<J, CT, 3>(p, ntiles, s);
    return launch_backward_k<J, CT, 2>(p, ntiles, s);
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
    const float unit =
        kIsSE16<CT> ? se16_unit((int)se16_expo<C>(p.coeff, (int64_t)p.g.width * p.g.height)[px] - kSE16Bias) : 0.f;
    auto bin = [&](int m) {
        float A = from_storage<CT>(c[0], 0, unit);
#pragma unroll
        for (int n = 0; n < J; ++n) {
            const int i = (1 << n) + (m >> (J - n));
            const float d = sqrt2_pow(n) * from_storage<CT>(c[i], i, unit);
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

template <int J, typename CT, int MB> cudaError_t launch_build_k(const Params &p, int ntiles, cudaStream_t s) {
    const int npx = p.g.tile_w * p.g.tile_h;
    const size_t bytes = Layout<J>::build(npx);
    if (bytes > kMaxSmemPerBlock) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(k_build<J, CT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_build<J, CT, MB><<<ntiles, kThreads, bytes, s>>>(p);
    return cudaGetLastError();
}
template <int J, typename CT> cudaError_t launch_build_t(const Params &p, int ntiles, cudaStream_t s) {
    if constexpr (J == 5) {
        if (p.g.tile_w * p.g.tile_h <= 192) return launch_build_k<J, CT, 4>(p, ntiles, s);
    }
    return launch_build_k<J, CT, MinBlocks<J>::value>(p, ntiles, s);
}

template <int J, typename CT, bool COMPOSITE, bool DEF, int MB>
cudaError_t launch_resolve_k(const Params &p, int ntiles, cudaStream_t s) {
    const int npx = p.g.tile_w * p.g.tile_h;
    const size_t bytes = Layout<J>::resolve(npx);
    if (bytes > kMaxSmemPerBlock) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(k_resolve<J, CT, COMPOSITE, DEF, MB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_resolve<J, CT, COMPOSITE, DEF, MB><<<ntiles, kThreads, bytes, s>>>(p);
    return cudaGetLastError();
}
// The accumulating resolve keeps one generic build; the compositing resolve
// (the second pass of the two-pass method) gets the default-flags and
// four-blocks builds of k_fused.
template <int J, typename CT, bool COMPOSITE>
cudaError_t launch_resolve_t(const Params &p, int ntiles, cudaStream_t s) {
    if constexpr (COMPOSITE) {
        const bool def = (p.flags & ~kAccumulate) == kDefaultFlags;
        if constexpr (J == 5) {
            if (p.g.tile_w * p.g.tile_h <= 192)
                return def ? launch_resolve_k<J, CT, true, true, 4>(p, ntiles, s)
                           : launch_resolve_k<J, CT, true, false, 4>(p, ntiles, s);
        }
        return def ? launch_resolve_k<J, CT, true, true, MinBlocks<J>::value>(p, ntiles, s)
                   : launch_resolve_k<J, CT, true, false, MinBlocks<J>::value>(p, ntiles, s);
    } else {
        return launch_resolve_k<J, CT, false, false, MinBlocks<J>::value>(p, ntiles, s);
    }
}

template <int J, typename CT, bool DEF, int MB>
cudaError_t launch_fused_k(const Params &p, int ntiles, cudaStream_t s) {
    const int npx = p.g.tile_w * p.g.tile_h;
    const size_t bytes = Layout<J>::fused(npx);
    if (bytes > kMaxSmemPerBlock) return cudaErrorNotSupported;
    cudaError_t e =
        cudaFuncSetAttribute(k_fused<J, CT, DEF, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_fused<J, CT, DEF, MB><<<ntiles, kThreads, bytes, s>>>(p);
    return cudaGetLastError();
}
template <int J, typename CT> cudaError_t launch_fused_t(const Params &p, int ntiles, cudaStream_t s) {
    const bool def = p.flags == kDefaultFlags;
    if constexpr (J == 5) {
        if (p.g.tile_w * p.g.tile_h <= kFourBlockTilePx)
            return def ? launch_fused_k<J, CT, true, 4>(p, ntiles, s) : launch_fused_k<J, CT, false, 4>(p, ntiles, s);
    }
    return def ? launch_fused_k<J, CT, true, MinBlocks<J>::value>(p, ntiles, s)
               : launch_fused_k<J, CT, false, MinBlocks<J>::value>(p, ntiles, s);
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
#define WT_JS(F, ...) {F<1, __VA_ARGS__>, F<2, __VA_ARGS__>, F<3, __VA_ARGS__>, F<4, __VA_ARGS__>, \
                       F<5, __VA_ARGS__>, F<6, __VA_ARGS__>}
#define WT_INSTANTIATE_TABLES(CT, IDX)                                                             \
    namespace wt {                                                                                \
    const TileLaunch kBuild##IDX[kMaxJ] = WT_JS(launch_build_t, CT);                               \
    const TileLaunch kResolve##IDX[kMaxJ] = WT_JS(launch_resolve_t, CT, false);                    \
    const TileLaunch kResolveComp##IDX[kMaxJ] = WT_JS(launch_resolve_t, CT, true);                 \
    const TileLaunch kFused##IDX[kMaxJ] = WT_JS(launch_fused_t, CT);                               \
    const TileLaunch kBackward##IDX[kMaxJ] = WT_JS(launch_backward_t, CT);                         \
    const ServeLaunch kServe##IDX[kMaxJ] = WT_JS(launch_serve_t, CT);                              \
    const ServeOccupancy kServeOcc##IDX[kMaxJ] = WT_JS(serve_blocks_per_sm, CT);                   \
    const TemporalLaunch kTemporal##IDX[kMaxJ] = WT_JS(launch_temporal_t, CT);                     \
    const QueryLaunch kAbsorbance##IDX[kMaxJ] = WT_JS(launch_absorbance_t, CT);                    \
    }
