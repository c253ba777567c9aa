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
// Each channel runs the mono kernel's phases in its shared memory: the
// channel's bins (fixed-point shared atomics, with the counting fallback), its
// coefficients and their storage, its bin values, and a resolve pass that
// accumulates (col_c w, w) per pixel.  With FP32 storage the channels are
// three launches of a one-channel kernel (mono-shaped: the mono kernel's
// register budget, four CTAs per SM); each writes its component of out and
// adds its coverage to out.w in channel order.  With E5B9G9R9 storage a word
// holds one coefficient index of all three channels, so one CTA per tile
// builds channels r and g first and keeps them until channel b is built; then
// the words are formed and stored, and the three resolves run on the decoded
// values, so that the composite matches the stored words.  Channels r and g
// wait as FP32 rows in shared memory when no word buffer is given
// (k_fused_rgb), and as 16-bit magnitudes in the word buffer itself when it is
// (k_fused_e5, half the shared memory).
#include "wt.h"
#include "wt_internal.h"
#include "wt_tile.cuh"

namespace wt {
namespace {

constexpr int kCh = 3;

struct RgbParams {
    Params p;  // geometry, fragments (pixel, z, r, g, b), coeff (nullable), out, bg, err
    const float *__restrict__ alpha_c[kCh];
    int64_t plane;  // P * C: stride of the FP32 channel planes
    int ch;         // FP32 storage: the channel of this launch
};

// Shared memory (bytes).  The region holds a channel's F and G bins, then its
// bin values followed by the staged coefficient rows, which are cleared and
// reused as the warps' (R, W) accumulators.  E5B9G9R9 adds the FP32 rows of
// channels r and g and one nearest-depth array per channel.
template <int J, bool E5> struct RgbLayout {
    static constexpr size_t rows(int npx) { return align16((size_t)npx * Shape<J>::C * 4); }
    static constexpr size_t accw(int npx) { return (size_t)kWarps * npx * 8; }
    static constexpr size_t after(int npx) { return rows(npx) > accw(npx) ? rows(npx) : accw(npx); }
    static constexpr size_t region(int npx) {
        return 2 * Layout<J>::plane(npx) > Layout<J>::vplane(npx) + after(npx) ? 2 * Layout<J>::plane(npx)
                                                                                : Layout<J>::vplane(npx) + after(npx);
    }
    static constexpr size_t stash(int npx) { return E5 ? 2 * rows(npx) : 0; }
    static constexpr size_t zw(int npx) { return region(npx) + stash(npx); }
    static constexpr size_t total(int npx) { return zw(npx) + (E5 ? kCh : 1) * Layout<J>::words(npx); }
};

// warp_accumulate on (R, W) pairs: the lanes holding the same pixel are
// ranked and add into the warp's private copy in rank order.
__device__ __forceinline__ void warp_accumulate2(float2 *mine, int lp, float2 v) {
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    const unsigned rank = __popc(__match_any_sync(0xffffffffu, lp) & lt);
    auto add = [&]() {
        float2 o = mine[lp];
        o.x += v.x;
        o.y += v.y;
        mine[lp] = o;
    };
    if (lp >= 0 && rank == 0) add();
    __syncwarp();
    for (unsigned r = 1; __any_sync(0xffffffffu, lp >= 0 && rank >= r); ++r) {
        if (lp >= 0 && rank == r) add();
        __syncwarp();
    }
}

// Step 3 for one channel: pc.alpha is the channel's opacity and pc.r its
// colour component; per pixel (R, W) += (col w, w), w = alpha 2^-A'.
template <int J, bool DEF>
__device__ __forceinline__ void resolve_channel(const Params &pc, const Tile &T, const float *A2, float2 *accw) {
    constexpr int LDV = Shape<J>::LDV;
    const uint32_t flags = DEF ? kDefaultFlags : pc.flags;
    const int npx = pc.g.tile_w * pc.g.tile_h;
    float2 *mine = accw + (threadIdx.x >> 5) * npx;
    for_each_group<kWithZ | kWithR>(T.s, T.e, pc, [&](auto &G) {
        constexpr int N = std::remove_reference_t<decltype(G)>::size;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int lp = G.v && G.z[k] == G.z[k] && G.al[k] == G.al[k] ? local_pixel(G.px[k], pc, T) : -1;
            const int l = lp >= 0 ? lp : 0;  // an invalid lane evaluates pixel 0 and adds nothing
            const float ac = clamp_alpha(G.al[k]);
            const float Ah = absorbance_at<J>(A2 + l * LDV, clamp_depth(G.z[k]), -lg2(1.f - ac), flags);
            const float w = ac * ex2(-Ah);
            warp_accumulate2(mine, lp, make_float2(G.r[k] * w, w));
        }
    });
}

// E5B9G9R9 of one coefficient index k (the stored magnitudes are chi and -X);
// the channels' values are replaced by the decoded ones.
__device__ __forceinline__ uint32_t pack_index(int k, float &r, float &g, float &b) {
    const float sg = k == 0 ? 1.f : -1.f;
    const uint32_t w = e5_encode(sg * r, sg * g, sg * b);
    e5_decode(w, r, g, b);
    r *= sg;
    g *= sg;
    b *= sg;
    return w;
}

// Step 2 for one channel (opacity alpha): its coefficients into v and its
// total step into S for the pixel of thread lp, its nearest depths into z.
// Ends with every bin row read.
template <int J>
__device__ __forceinline__ void build_channel(const Params &p, const float *alpha, const Tile &T,
                                              unsigned char *smem, unsigned *z, int64_t gp,
                                              float (&v)[1 << J], float &S, unsigned &bad) {
    constexpr int LD = Shape<J>::LD;
    const int npx = p.g.tile_w * p.g.tile_h, lp = threadIdx.x;
    unsigned *sF = reinterpret_cast<unsigned *>(smem);
    unsigned *sG = reinterpret_cast<unsigned *>(smem + Layout<J>::plane(npx));
    Params pc = p;
    pc.alpha = alpha;
    fill_zero(smem, (int)(2 * Layout<J>::plane(npx)));
    for (int i = threadIdx.x; i < npx; i += blockDim.x) z[i] = 0x7f800000u;
    __syncthreads();
    const bool scaled = phase_bins<J>(pc, T, sF, sG, z, bad);
    if (gp >= 0) bins_to_coeffs<J>(sF + lp * LD, sG + lp * LD, v, S, scaled);
    __syncthreads();
}

// Steps 3 and 4 for one channel from its coefficients in v (the accumulators
// cleared by the caller): bin values, the resolve pass, and the channel's
// composite out of its sums, its total step S and its background bg.
template <int J, bool DEF>
__device__ __forceinline__ void resolve_channel_px(const Params &p, const float *alpha, const float *col,
                                                   const Tile &T, unsigned char *smem, const unsigned *z,
                                                   int64_t gp, float (&v)[1 << J], float S, float bg, float &o,
                                                   float &cover_sum) {
    constexpr int LDV = Shape<J>::LDV;
    const uint32_t flags = DEF ? kDefaultFlags : p.flags;
    const int npx = p.g.tile_w * p.g.tile_h, lp = threadIdx.x;
    float *vals = reinterpret_cast<float *>(smem);
    float2 *accw = reinterpret_cast<float2 *>(smem + Layout<J>::vplane(npx));
    if (gp >= 0) {
        coeffs_to_bins<J>(v, kLog2e);
        put_bins<J>(vals + lp * LDV, v, __uint_as_float(z[lp]), flags);
    }
    __syncthreads();
    Params pc = p;
    pc.alpha = alpha;
    pc.r = col;
    resolve_channel<J, DEF>(pc, T, vals, accw);
    __syncthreads();
    if (gp >= 0) {
        float2 a = accw[lp];
#pragma unroll
        for (int w = 1; w < kWarps; ++w) {
            const float2 u = accw[w * npx + lp];
            a.x += u.x;
            a.y += u.y;
        }
        const float Tc = ex2(-S * kLog2e);
        // 1 - T; for small S the series S (1 - S/2)
        const float cover = S < 0.0009765625f ? S * fmaf(-0.5f, S, 1.f) : 1.f - Tc;
        if (flags & kNormalized) {
            if (a.y > 0.f) {
                const float k = a.y >= 1.17549435e-38f ? cover * rcp(a.y) : cover / a.y;  // (subnormal W)
                o = fmaf(a.x, k, bg * Tc);
            } else {
                o = bg;
            }
        } else {
            o = fmaf(bg, Tc, a.x);
        }
        cover_sum += cover;
    }
    __syncthreads();  // accumulators read
}

template <int J, bool E5, bool DEF, int MB>
__global__ void __launch_bounds__(kThreads, MB) k_fused_rgb(RgbParams q) {
    constexpr int C = Shape<J>::C;
    using L = RgbLayout<J, E5>;
    using St = Staged<float, C>;
    extern __shared__ __align__(16) unsigned char smem[];
    const Params &p = q.p;
    const int npx = p.g.tile_w * p.g.tile_h;
    uint4 *stage = reinterpret_cast<uint4 *>(smem + Layout<J>::vplane(npx));  // rows out, then (R, W)
    const int after = (int)L::after(npx);
    const Tile T = tile_of(p, p.tile0 + (int)blockIdx.x, E5 || q.ch == 0);  // a bad range counts once
    const int lp = threadIdx.x;
    int64_t gp = -1;
    if (lp < npx) gp = global_pixel(p, T, lp);
    float v[C];
    unsigned bad = 0;
    auto bg_of = [&](int c) {
        return p.bg_img && gp >= 0 ? p.bg_img[3 * gp + c] : (c == 0 ? p.bg0 : c == 1 ? p.bg1 : p.bg2);
    };

    if constexpr (!E5) {
        // one channel per launch (the three launches share the mono kernel's
        // register budget and shared memory); its result goes to its component
        // of out, and its coverage is added to out.w in channel order
        const int c = q.ch;
        const float *alpha = c == 0 ? q.alpha_c[0] : c == 1 ? q.alpha_c[1] : q.alpha_c[2];
        const float *col = c == 0 ? p.r : c == 1 ? p.gc : p.b;
        if (threadIdx.x == 0) {
            l2_prefetch_range(p.pixel, T.s, T.e);
            l2_prefetch_range(p.z, T.s, T.e);
            l2_prefetch_range(alpha, T.s, T.e);
            l2_prefetch_range(col, T.s, T.e);
        }
        unsigned *sZ = reinterpret_cast<unsigned *>(smem + L::zw(npx));
        float S = 0.f;
        build_channel<J>(p, alpha, T, smem, sZ, gp, v, S, bad);
        float *dst = p.coeff ? static_cast<float *>(p.coeff) + c * q.plane : nullptr;
        if (dst && St::ok) {
            if (gp >= 0) stage_row<float, C>(stage, lp, v);
            __syncthreads();
            copy_staged<float, C>(p, T, stage, after, dst);  // clears the accumulators
        } else {
            if (dst && gp >= 0) store_row<float, C>(dst + gp * C, v);
            fill_zero(stage, after);
        }
        float oc = 0.f, cs = 0.f;
        resolve_channel_px<J, DEF>(p, alpha, col, T, smem, sZ, gp, v, S, bg_of(c), oc, cs);
        if (gp >= 0) {
            float *px = p.out + 4 * gp;
            px[c] = oc;
            px[3] = c == 0 ? cs : (c == 1 ? px[3] + cs : (px[3] + cs) * (1.f / 3.f));
        }
    } else {
        if (threadIdx.x == 0) {
            l2_prefetch_range(p.pixel, T.s, T.e);
            l2_prefetch_range(p.z, T.s, T.e);
#pragma unroll
            for (int c = 0; c < kCh; ++c) l2_prefetch_range(q.alpha_c[c], T.s, T.e);
            l2_prefetch_range(p.r, T.s, T.e);
            l2_prefetch_range(p.gc, T.s, T.e);
            l2_prefetch_range(p.b, T.s, T.e);
        }
        uint4 *stash0 = reinterpret_cast<uint4 *>(smem + L::region(npx));
        uint4 *stash1 = reinterpret_cast<uint4 *>(smem + L::region(npx) + L::rows(npx));
        const int zs = (int)(Layout<J>::words(npx) / 4);
        unsigned *sZ = reinterpret_cast<unsigned *>(smem + L::zw(npx));
        uint32_t *words = static_cast<uint32_t *>(p.coeff);
        float S[kCh] = {0.f, 0.f, 0.f}, o[kCh] = {0.f, 0.f, 0.f}, cover_sum = 0.f;
        build_channel<J>(p, q.alpha_c[0], T, smem, sZ, gp, v, S[0], bad);
        if (gp >= 0) {
            if constexpr (St::ok) stage_row<float, C>(stash0, lp, v);
            else for (int k = 0; k < C; ++k) reinterpret_cast<float *>(stash0)[lp * C + k] = v[k];
        }
        build_channel<J>(p, q.alpha_c[1], T, smem, sZ + zs, gp, v, S[1], bad);
        if (gp >= 0) {
            if constexpr (St::ok) stage_row<float, C>(stash1, lp, v);
            else for (int k = 0; k < C; ++k) reinterpret_cast<float *>(stash1)[lp * C + k] = v[k];
        }
        build_channel<J>(p, q.alpha_c[2], T, smem, sZ + 2 * zs, gp, v, S[2], bad);
        // the words, index by index; the decoded values replace the FP32 ones
        if (gp >= 0) {
            if constexpr (St::ok) {
                const int sw = St::sw(lp);
#pragma unroll
                for (int ch = 0; ch < St::K; ++ch) {
                    const int at = lp * St::K + (ch ^ sw);
                    float4 r = reinterpret_cast<const float4 *>(stash0)[at];
                    float4 g = reinterpret_cast<const float4 *>(stash1)[at];
                    uint4 w;
                    w.x = pack_index(4 * ch, r.x, g.x, v[4 * ch]);
                    w.y = pack_index(4 * ch + 1, r.y, g.y, v[4 * ch + 1]);
                    w.z = pack_index(4 * ch + 2, r.z, g.z, v[4 * ch + 2]);
                    w.w = pack_index(4 * ch + 3, r.w, g.w, v[4 * ch + 3]);
                    reinterpret_cast<float4 *>(stash0)[at] = r;
                    reinterpret_cast<float4 *>(stash1)[at] = g;
                    if (words) stage[at] = w;
                }
            } else {
                float *r = reinterpret_cast<float *>(stash0) + lp * C;
                float *g = reinterpret_cast<float *>(stash1) + lp * C;
#pragma unroll
                for (int k = 0; k < C; ++k) {
                    const uint32_t w = pack_index(k, r[k], g[k], v[k]);
                    if (words) words[gp * C + k] = w;
                }
            }
        }
        if (words && St::ok) {
            __syncthreads();
            copy_staged<float, C>(p, T, stage, after, reinterpret_cast<float *>(words));
        } else {
            fill_zero(stage, after);
        }
        resolve_channel_px<J, DEF>(p, q.alpha_c[2], p.b, T, smem, sZ + 2 * zs, gp, v, S[2], bg_of(2), o[2],
                                   cover_sum);
#pragma unroll
        for (int c = 1; c >= 0; --c) {
            if (gp >= 0) {
                const uint4 *src = c == 0 ? stash0 : stash1;
                if constexpr (St::ok) unstage_row<float, C>(src, lp, v);
                else for (int k = 0; k < C; ++k) v[k] = reinterpret_cast<const float *>(src)[lp * C + k];
            }
            fill_zero(stage, after);
            resolve_channel_px<J, DEF>(p, q.alpha_c[c], c == 0 ? p.r : p.gc, T, smem, sZ + c * zs, gp, v, S[c],
                                       bg_of(c), o[c], cover_sum);
        }
        if (gp >= 0) reinterpret_cast<float4 *>(p.out)[gp] = make_float4(o[0], o[1], o[2], cover_sum * (1.f / 3.f));
    }
    flush_bad(bad, p.err);
}

// A clamped channel magnitude y in [0, kE5Max] kept in 16 bits for the word
// formation: 0 for y < 2^-25, else its FP32 exponent E in [-25, 15] (6 bits, as
// E + 26) and the top 10 bits of its mantissa, i.e. t = (bits(y) - bits(2^-26))
// >> 13.  The word reads no more of y: its shared exponent comes from the
// largest value's exponent and its 9-bit mantissa (rounded), which are the
// top 10 significant bits at most, and every other channel's mantissa
// floor(y 2^(24 - e) + 1/2) is fixed by the bits of y down to 2^(e - 25),
// again 10 significant bits at most (e >= floor(log2 y) + 16).  Below 2^-25
// a value has mantissa 0 in every word and cannot raise the exponent, whose
// floor is -16.  So the words formed from the 16-bit values are the words of
// the FP32 values, bit for bit.
__device__ __forceinline__ uint32_t e5_keep16(float y) {
    const uint32_t u = __float_as_uint(y);
    return u < 0x33000000u ? 0u : (u - 0x32800000u) >> 13;  // 2^-25, 2^-26
}
__device__ __forceinline__ float e5_from16(uint32_t t) { return t ? __uint_as_float((t << 13) + 0x32800000u) : 0.f; }

// Channel c (0 or 1) of a pixel's coefficient row v, as the magnitudes the
// words encode (chi_00 and -X), in 16 bits each: half c of the pixel's row of
// words (C / 2 words), which is free until the words are formed.
template <int C> __device__ __forceinline__ void stash16(uint32_t *row, int c, const float (&v)[C]) {
    uint32_t h[C / 2];
#pragma unroll
    for (int i = 0; i < C / 2; ++i) {
        const float a = e5_clamp(i == 0 ? v[0] : -v[2 * i]), b = e5_clamp(-v[2 * i + 1]);
        h[i] = e5_keep16(a) | (e5_keep16(b) << 16);
    }
    uint32_t *dst = row + c * (C / 2);
    if constexpr (C / 2 % 4 == 0) {
#pragma unroll
        for (int i = 0; i < C / 2; i += 4)
            reinterpret_cast<uint4 *>(dst)[i / 4] = make_uint4(h[i], h[i + 1], h[i + 2], h[i + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < C / 2; ++i) dst[i] = h[i];
    }
}
template <int C> __device__ __forceinline__ float unstash16(const uint32_t *row, int c, int k) {
    const uint32_t h = row[c * (C / 2) + k / 2];
    return e5_from16(k & 1 ? h >> 16 : h & 0xffffu);
}

// E5B9G9R9 storage with the word buffer given.  The channels run one after
// another through the one-channel kernel's phases and shared memory (one
// nearest-depth array: 57 KB at J = 5 with 192-pixel tiles, three blocks per
// SM as the registers allow, against two for the two-rows kernel above):
//   * r and g: bins, coefficients; the coefficients go, as 16-bit magnitudes,
//     into halves of the pixel's own row of words, and the nearest depth and
//     total step into the pixel's out entry (both read back by the same thread);
//   * b: bins, coefficients, then the words from the stashed r, g and b, and
//     the resolve of b on its decoded values;
//   * g, then r: the channel decoded from the stored words, its nearest depth
//     and total step from out, and its resolve.
// Every value reaches the same arithmetic as in the two-rows kernel above, so
// words and composite are bit for bit the same.
template <int J, bool DEF, int MB>
__global__ void __launch_bounds__(kThreads, MB) k_fused_e5(RgbParams q) {
    constexpr int C = Shape<J>::C;
    using L = RgbLayout<J, false>;
    using St = Staged<float, C>;
    extern __shared__ __align__(16) unsigned char smem[];
    const Params &p = q.p;
    const int npx = p.g.tile_w * p.g.tile_h;
    uint4 *stage = reinterpret_cast<uint4 *>(smem + Layout<J>::vplane(npx));  // words out, then (R, W)
    const int after = (int)L::after(npx);
    const Tile T = tile_of(p, p.tile0 + (int)blockIdx.x, true);
    const int lp = threadIdx.x;
    int64_t gp = -1;
    if (lp < npx) gp = global_pixel(p, T, lp);
    uint32_t *words = static_cast<uint32_t *>(p.coeff);
    uint32_t *row = words + (gp >= 0 ? gp : 0) * C;
    float2 *keep = reinterpret_cast<float2 *>(p.out) + 2 * (gp >= 0 ? gp : 0);  // (zmin, S) of r, then g
    unsigned *sZ = reinterpret_cast<unsigned *>(smem + L::zw(npx));
    if (threadIdx.x == 0) {
        l2_prefetch_range(p.pixel, T.s, T.e);
        l2_prefetch_range(p.z, T.s, T.e);
#pragma unroll
        for (int c = 0; c < kCh; ++c) l2_prefetch_range(q.alpha_c[c], T.s, T.e);
        l2_prefetch_range(p.r, T.s, T.e);
        l2_prefetch_range(p.gc, T.s, T.e);
        l2_prefetch_range(p.b, T.s, T.e);
    }
    auto bg_of = [&](int c) {
        return p.bg_img && gp >= 0 ? p.bg_img[3 * gp + c] : (c == 0 ? p.bg0 : c == 1 ? p.bg1 : p.bg2);
    };
    // (each phase has its own coefficient array, which a thread outside the
    // image leaves unset, so that no array stays live across a bins pass)
    unsigned bad = 0;
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
        float v[C], S = 0.f;
        build_channel<J>(p, c == 0 ? q.alpha_c[0] : q.alpha_c[1], T, smem, sZ, gp, v, S, bad);
        if (gp >= 0) {
            stash16<C>(row, c, v);
            keep[c] = make_float2(__uint_as_float(sZ[lp]), S);
        }
    }
    float ob = 0.f, og = 0.f, orr = 0.f, cover_sum = 0.f;
    {
    float v[C], S = 0.f;
    build_channel<J>(p, q.alpha_c[2], T, smem, sZ, gp, v, S, bad);
    // the words; channel b's decoded values replace its FP32 ones
    if constexpr (St::ok) {
        // b's rows staged in the free bins region; then one 4-index chunk of one
        // pixel per item: the two stashed halves, b, four words (staged for the
        // coalesced copy), b decoded in place
        uint4 *bst = reinterpret_cast<uint4 *>(smem);
        if (gp >= 0) stage_row<float, C>(bst, lp, v);
        __syncthreads();
        for (int it = threadIdx.x; it < npx * St::K; it += blockDim.x) {
            const int l = it / St::K, ch = it % St::K;
            const int64_t g2 = global_pixel(p, T, l);
            if (g2 < 0) continue;
            const uint32_t *r2 = words + g2 * C;
            const uint2 hr = reinterpret_cast<const uint2 *>(r2)[ch];
            const uint2 hg = reinterpret_cast<const uint2 *>(r2 + C / 2)[ch];
            const int at = l * St::K + (ch ^ St::sw(l));
            float4 b = reinterpret_cast<const float4 *>(bst)[at];
            auto word = [&](uint32_t r16, uint32_t g16, float &x, float sg) {
                const uint32_t w = e5_encode(e5_from16(r16), e5_from16(g16), sg * x);
                float dr, dg, db;
                e5_decode(w, dr, dg, db);
                x = sg * db;
                return w;
            };
            uint4 w;
            w.x = word(hr.x & 0xffffu, hg.x & 0xffffu, b.x, ch == 0 ? 1.f : -1.f);
            w.y = word(hr.x >> 16, hg.x >> 16, b.y, -1.f);
            w.z = word(hr.y & 0xffffu, hg.y & 0xffffu, b.z, -1.f);
            w.w = word(hr.y >> 16, hg.y >> 16, b.w, -1.f);
            reinterpret_cast<float4 *>(bst)[at] = b;
            stage[at] = w;
        }
        __syncthreads();  // every stash read before any row is overwritten
        copy_staged<float, C>(p, T, stage, after, reinterpret_cast<float *>(words));
        if (gp >= 0) unstage_row<float, C>(bst, lp, v);
        __syncthreads();  // b's rows read before its bin values overwrite them
    } else {
        if (gp >= 0) {
            uint32_t w[C];
#pragma unroll
            for (int k = 0; k < C; ++k) {
                const float sg = k == 0 ? 1.f : -1.f;
                w[k] = e5_encode(unstash16<C>(row, 0, k), unstash16<C>(row, 1, k), sg * v[k]);
                float dr, dg, db;
                e5_decode(w[k], dr, dg, db);
                v[k] = sg * db;
            }
#pragma unroll
            for (int k = 0; k < C; ++k) row[k] = w[k];  // every stash read before the row is overwritten
        }
        fill_zero(stage, after);
    }
    resolve_channel_px<J, DEF>(p, q.alpha_c[2], p.b, T, smem, sZ, gp, v, S, bg_of(2), ob, cover_sum);
    }
    // (its barriers have made every word of the tile visible to the block)
#pragma unroll 1
    for (int c = 1; c >= 0; --c) {
        float v[C], Sc = 0.f, oc = 0.f;
        if (gp >= 0) {
            const float2 zs = keep[c];
            sZ[lp] = __float_as_uint(zs.x);
            Sc = zs.y;
            auto take = [&](int k, uint32_t w) {
                float r, g, b;
                e5_decode(w, r, g, b);
                v[k] = (k == 0 ? 1.f : -1.f) * (c == 0 ? r : g);
            };
            if constexpr (C % 4 == 0) {
#pragma unroll
                for (int k = 0; k < C; k += 4) {
                    const uint4 w = reinterpret_cast<const uint4 *>(row)[k / 4];
                    take(k, w.x);
                    take(k + 1, w.y);
                    take(k + 2, w.z);
                    take(k + 3, w.w);
                }
            } else {
#pragma unroll
                for (int k = 0; k < C; ++k) take(k, row[k]);
            }
        }
        fill_zero(stage, after);
        resolve_channel_px<J, DEF>(p, c == 0 ? q.alpha_c[0] : q.alpha_c[1], c == 0 ? p.r : p.gc, T, smem, sZ,
                                   gp, v, Sc, bg_of(c), oc, cover_sum);
        if (c == 0) orr = oc;
        else og = oc;
    }
    if (gp >= 0) reinterpret_cast<float4 *>(p.out)[gp] = make_float4(orr, og, ob, cover_sum * (1.f / 3.f));
    flush_bad(bad, p.err);
}

// FP32 storage uses the mono kernel's shared memory and register budget (four
// blocks per SM at J = 5 with 192-pixel tiles); E5B9G9R9 keeps two more
// coefficient rows per pixel and takes fewer blocks.
template <int J, bool E5, bool DEF> cudaError_t launch_rgb(const RgbParams &q, int ntiles, cudaStream_t s) {
    constexpr int MB = E5 ? (J == 5 ? 2 : 3) : 4;
    const int npx = q.p.g.tile_w * q.p.g.tile_h;
    const size_t bytes = RgbLayout<J, E5>::total(npx);
    if (bytes > kMaxSmemPerBlock) return cudaErrorNotSupported;
    cudaError_t e =
        cudaFuncSetAttribute(k_fused_rgb<J, E5, DEF, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_fused_rgb<J, E5, DEF, MB><<<ntiles, kThreads, bytes, s>>>(q);
    return cudaGetLastError();
}

// E5B9G9R9 with the word buffer given: the one-channel kernel's shared memory;
// registers for three blocks per SM from J = 3 on (at 64 registers the three
// channels' phases spill: 400 bytes per thread at J = 5, measured 8.96 ms
// against 8.33 ms at three blocks).
template <int J, bool DEF> cudaError_t launch_e5(const RgbParams &q, int ntiles, cudaStream_t s) {
    constexpr int MB = J >= 3 ? 3 : 4;
    const int npx = q.p.g.tile_w * q.p.g.tile_h;
    const size_t bytes = RgbLayout<J, false>::total(npx);
    if (bytes > kMaxSmemPerBlock) return cudaErrorNotSupported;
    cudaError_t e =
        cudaFuncSetAttribute(k_fused_e5<J, DEF, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_fused_e5<J, DEF, MB><<<ntiles, kThreads, bytes, s>>>(q);
    return cudaGetLastError();
}

typedef cudaError_t (*RgbLaunch)(const RgbParams &, int, cudaStream_t);
#define WT_RGB_ROW(E5, DEF) \
    { launch_rgb<1, E5, DEF>, launch_rgb<2, E5, DEF>, launch_rgb<3, E5, DEF>, launch_rgb<4, E5, DEF>, launch_rgb<5, E5, DEF> }
const RgbLaunch kRgb[2][2][5] = {{WT_RGB_ROW(false, false), WT_RGB_ROW(false, true)},
                                 {WT_RGB_ROW(true, false), WT_RGB_ROW(true, true)}};
#undef WT_RGB_ROW
#define WT_E5_ROW(DEF) { launch_e5<1, DEF>, launch_e5<2, DEF>, launch_e5<3, DEF>, launch_e5<4, DEF>, launch_e5<5, DEF> }
const RgbLaunch kE5[2][5] = {WT_E5_ROW(false), WT_E5_ROW(true)};
#undef WT_E5_ROW

template <int J> size_t rgb_bytes(int npx, bool e5) {
    return e5 ? RgbLayout<J, true>::total(npx) : RgbLayout<J, false>::total(npx);
}

}  // namespace

// Shared memory the coloured kernel needs for a tile of npx pixels at J.
size_t rgb_smem_bytes(int J, int npx, bool e5) {
    switch (J) {
    case 1: return rgb_bytes<1>(npx, e5);
    case 2: return rgb_bytes<2>(npx, e5);
    case 3: return rgb_bytes<3>(npx, e5);
    case 4: return rgb_bytes<4>(npx, e5);
    default: return rgb_bytes<5>(npx, e5);
    }
}

cudaError_t launch_fused_rgb(const Params &p, int J, const float *const alpha_c[3], bool e5, int ntiles,
                             cudaStream_t s) {
    RgbParams q;
    q.p = p;
    for (int c = 0; c < kCh; ++c) q.alpha_c[c] = alpha_c[c];
    q.plane = (int64_t)p.g.width * p.g.height * (int64_t(1) << J);
    const int def = p.flags == kDefaultFlags ? 1 : 0;
    const RgbLaunch f = kRgb[e5 ? 1 : 0][def][J - 1];
    if (e5) {
        q.ch = 0;
        return (p.coeff ? kE5[def][J - 1] : f)(q, ntiles, s);
    }
    for (int c = 0; c < kCh; ++c) {
        q.ch = c;
        const cudaError_t e = f(q, ntiles, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace wt
