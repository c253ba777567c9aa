// Device-side building blocks of the Wavelet OIT kernels (sm_103a).
//
// One CTA owns one screen tile (<= 256 pixels, one thread per pixel in the
// per-pixel phases).  The tile's fragments are a contiguous range of the
// tile-grouped stream, read with 16-byte vector loads.  Fragments of the same
// pixel meet in shared memory (the coefficient update of §2.3.3), never in
// global atomics.
//
// Build.  Instead of touching J+1 coefficients per fragment, every fragment
// adds (a f, a (1-f)) to one bin of its pixel at the finest level
// (bin m = floor(C z), fraction f = C z - m):
//     F_m = sum a_i f_i,      G_m = sum a_i (1 - f_i),
// and an O(C) tree per pixel turns the bins into the coefficients of §2.3.1.
// The bins are 32-bit fixed point with a per-pixel power-of-two scale s_p
// chosen by a counting pass (c_p fragments whose largest step is a_max give
// c_p a_max s_p <= 2^31, so no bin can overflow), and are added with integer
// atomics: the sums do not depend on the order of the fragments, so the
// coefficients -- and everything computed from them in one CTA -- are the
// same on every run, alone or batched with other frames.
// For a dyadic interval I with children L, R and u the position normalised to
// I, F_I = sum_I a u and G_I = sum_I a (1-u) satisfy
//     t = F_L + G_R,   F_I = t/2 + F_R,   G_I = t/2 + G_L,
//     sum_I a Psi_{n,k} = 2^{-n/2} t / 2      (Psi is u then 1-u, scaled),
// so X_{n,k} = -2^{-n/2} t / 2, chi_00 = G_root and sum a = F_root + G_root.
// Every quantity is a sum of non-negative terms (no cancellation in FP32).
//
// Resolve.  The coefficients are synthesised once per pixel into the C bin
// values at the bin centres (§2.3.2), kept in shared memory pre-multiplied by
// log2(e), so a fragment's transmittance is one ex2 instruction.
//
// The build's bins take FP32 shared-memory atomic adds (separate F and G
// planes, so a warp's lanes spread over the banks).  The resolve's per-pixel
// sums use a warp-segmented reduction instead of atomics: the lanes of a warp
// that hold the same pixel are grouped (match.any), the group's leader adds
// its peers' values through shuffles and applies one plain read-modify-write
// to the warp's private copy of the accumulators; the copies are summed per
// pixel at the end of the tile.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wt {

constexpr int kThreads = 256;    // threads per CTA (= max pixels per tile)
constexpr int kMaxTilePx = 256;
constexpr int kWarps = kThreads / 32;  // warp-private copies of the per-pixel accumulators
constexpr int kCasLimit = 1 << 20;  // bound on CAS retries (never reached in practice)
// alpha is clamped to [0, 1 - 2^-20] and z to [0, 1 - 2^-24] (exact in FP32)
constexpr float kAlphaMax = 0.99999904632568359375f;
constexpr float kZMax = 0.999999940395355224609375f;
constexpr float kLog2e = 1.44269504088896340736f;
// the largest step after the clamp is -ln(2^-20) = 20 ln 2, i.e. 20 in log2 units
constexpr float kStepCapLog2 = 20.0f;

struct Geom {
    int width, height, tile_w, tile_h, ntx;
};

// Everything a kernel reads or writes; passed by value.
struct Params {
    Geom g;
    uint32_t flags;
    uint64_t wmagic;  // floor((2^64-1) / width) + 1 for the division by width (0 when width == 1)
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
    // adjoint: dL/d(out) [P*4] in, dL/dalpha [n] and dL/d(r,g,b) [3*n] out
    const float *__restrict__ gout;
    float *galpha;
    float *grgb;
};

enum : uint32_t { kSelfExclude = 1u, kLinear = 2u, kNormalized = 4u, kAccumulate = 8u };

template <int J> struct Shape {
    static constexpr int C = 1 << J;
    static constexpr int LD = C + 4;  // words per pixel row of bins / bin values (16-byte rows)
    // the padding words of a pixel's F row hold its counting-pass results
    static constexpr int CNT = C, AMAX = C + 1, INV = C + 2;
};

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

// One pixel's C coefficients to / from global memory, 16-byte vectors when
// the row is a multiple of 16 bytes (it is 16-byte aligned then).
template <typename CT, int C>
__device__ __forceinline__ void store_row(CT *dst, const float (&v)[C]) {
    constexpr int PER = 16 / sizeof(CT);
    if constexpr (C % PER == 0) {
#pragma unroll
        for (int q = 0; q < C / PER; ++q) {
            union { uint4 u; CT e[PER]; } pk;
#pragma unroll
            for (int i = 0; i < PER; ++i) pk.e[i] = Cvt<CT>::to(v[q * PER + i]);
            reinterpret_cast<uint4 *>(dst)[q] = pk.u;
        }
    } else {
#pragma unroll
        for (int i = 0; i < C; ++i) dst[i] = Cvt<CT>::to(v[i]);
    }
}

template <typename CT, int C>
__device__ __forceinline__ void load_row(const CT *src, float (&v)[C]) {
    constexpr int PER = 16 / sizeof(CT);
    if constexpr (C % PER == 0) {
#pragma unroll
        for (int q = 0; q < C / PER; ++q) {
            union { uint4 u; CT e[PER]; } pk;
            pk.u = reinterpret_cast<const uint4 *>(src)[q];
#pragma unroll
            for (int i = 0; i < PER; ++i) v[q * PER + i] = Cvt<CT>::from(pk.e[i]);
        }
    } else {
#pragma unroll
        for (int i = 0; i < C; ++i) v[i] = Cvt<CT>::from(src[i]);
    }
}

// ---------------------------------------------------------------- tiles

struct Tile {
    int tx0, ty0, tw, th;  // origin and clipped extent
    uint32_t base, lim;    // pixel id of the tile origin; th * width
    int64_t s, e;          // fragment range
};

__device__ __forceinline__ Tile tile_of(const Params &p, int t, bool count_bad) {
    Tile T;
    const int tx = t % p.g.ntx, ty = t / p.g.ntx;
    T.tx0 = tx * p.g.tile_w;
    T.ty0 = ty * p.g.tile_h;
    T.tw = min(p.g.tile_w, p.g.width - T.tx0);
    T.th = min(p.g.tile_h, p.g.height - T.ty0);
    T.base = (uint32_t)T.ty0 * (uint32_t)p.g.width + (uint32_t)T.tx0;
    T.lim = (uint32_t)T.th * (uint32_t)p.g.width;
    int64_t s = p.off[t], e = p.off[t + 1];
    if (s < 0 || e < s || e > p.n) {  // corrupt range: skip the tile, count once
        if (count_bad && threadIdx.x == 0) atomicAdd(p.err, 1ull);
        s = e = 0;
    }
    T.s = s;
    T.e = e;
    return T;
}

// Local pixel index inside the tile, or -1 when the pixel is not in it.
// d = pixel - tile origin; its row is d / width, taken as the high word of
// d * ceil(2^64 / width) (exact for 32-bit d; Granlund & Montgomery 1994).
__device__ __forceinline__ int local_pixel(uint32_t px, const Params &p, const Tile &T) {
    const uint32_t d = px - T.base;
    if (d >= T.lim) return -1;
    const uint32_t ly = p.wmagic ? (uint32_t)__umul64hi((uint64_t)d, p.wmagic) : d;
    const uint32_t lx = d - ly * (uint32_t)p.g.width;
    if (lx >= (uint32_t)T.tw) return -1;
    return (int)(ly * (uint32_t)p.g.tile_w + lx);
}

// global pixel id of local pixel lp, or -1 if it lies outside the image
__device__ __forceinline__ int64_t global_pixel(const Params &p, const Tile &T, int lp) {
    const int lx = lp % p.g.tile_w, ly = lp / p.g.tile_w;
    if (lx >= T.tw || ly >= T.th) return -1;
    return (int64_t)(T.ty0 + ly) * p.g.width + T.tx0 + lx;
}

// ---------------------------------------------------------------- conditioning

__device__ __forceinline__ float clamp_alpha(float al) { return fminf(fmaxf(al, 0.f), kAlphaMax); }
__device__ __forceinline__ float clamp_depth(float z) { return fminf(fmaxf(z, 0.f), kZMax); }
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Absorbance step of one interface, a = -ln(1 - x) for x = clamped alpha
// (v drops by the factor 1 - alpha across it).
//  x <= 1/2: -ln(1 - x) = 2 atanh(s) with s = x / (2 - x) <= 1/3, summed as
//            the odd power series 2 s (1 + s^2/3 + ... + s^12/13); the first
//            omitted term is below 2e-8 relative.
//  x >  1/2: 1 - x is exact in FP32 (Sterbenz), its log2 is >= 1 in magnitude,
//            so the hardware log2 (relative error ~2^-22) suffices.
// Checked against log1p in FP64 to a few ulp over the whole clamped range.
__device__ __forceinline__ float step_of(float x) {
    const float s = x * rcp(2.f - x);
    const float s2 = s * s;
    float q = fmaf(s2, 1.f / 13, 1.f / 11);
    q = fmaf(s2, q, 1.f / 9);
    q = fmaf(s2, q, 1.f / 7);
    q = fmaf(s2, q, 1.f / 5);
    q = fmaf(s2, q, 1.f / 3);
    q = fmaf(s2, q, 1.f);
    const float series = 2.f * s * q;
    const float direct = -0.693147180559945309f * lg2(1.f - x);
    return x <= 0.5f ? series : direct;
}

// ---------------------------------------------------------------- streaming

// Calls body(pixel, alpha) for every fragment of [s, e), 4 per 16-byte load.
template <class Body>
__device__ __forceinline__ void for_each_frag2(int64_t s, int64_t e, const Params &p, Body &&body) {
    const int tid = threadIdx.x, nt = blockDim.x;
    int64_t s4 = (s + 3) & ~int64_t(3), e4 = e & ~int64_t(3);
    if (s4 > e4) s4 = e4 = e;
    for (int64_t i = s + tid; i < s4; i += nt) body(p.pixel[i], p.alpha[i]);
    const uint4 *px4 = reinterpret_cast<const uint4 *>(p.pixel);
    const float4 *a4 = reinterpret_cast<const float4 *>(p.alpha);
    for (int64_t q = (s4 >> 2) + tid; q < (e4 >> 2); q += nt) {
        const uint4 pv = px4[q];
        const float4 av = a4[q];
        body(pv.x, av.x);
        body(pv.y, av.y);
        body(pv.z, av.z);
        body(pv.w, av.w);
    }
    for (int64_t i = e4 + tid; i < e; i += nt) body(p.pixel[i], p.alpha[i]);
}

// Calls body(pixel, z, alpha) for every fragment of [s, e), 4 per 16-byte load;
// the loads of the next chunk are issued before the current one is processed.
template <class Body>
__device__ __forceinline__ void for_each_frag3(int64_t s, int64_t e, const Params &p, Body &&body) {
    const int tid = threadIdx.x, nt = blockDim.x;
    int64_t s4 = (s + 3) & ~int64_t(3), e4 = e & ~int64_t(3);
    if (s4 > e4) s4 = e4 = e;
    for (int64_t i = s + tid; i < s4; i += nt) body(p.pixel[i], p.z[i], p.alpha[i]);
    const uint4 *px4 = reinterpret_cast<const uint4 *>(p.pixel);
    const float4 *z4 = reinterpret_cast<const float4 *>(p.z);
    const float4 *a4 = reinterpret_cast<const float4 *>(p.alpha);
    {
        const int64_t qe = e4 >> 2;
        int64_t q = (s4 >> 2) + tid;
        uint4 pv = make_uint4(0, 0, 0, 0);
        float4 zv = make_float4(0.f, 0.f, 0.f, 0.f), av = zv;
        if (q < qe) {
            pv = px4[q];
            zv = z4[q];
            av = a4[q];
        }
        while (q < qe) {
            const uint4 cp = pv;
            const float4 cz = zv, ca = av;
            const int64_t qn = q + nt;
            if (qn < qe) {  // next chunk in flight while this one is processed
                pv = px4[qn];
                zv = z4[qn];
                av = a4[qn];
            }
            body(cp.x, cz.x, ca.x);
            body(cp.y, cz.y, ca.y);
            body(cp.z, cz.z, ca.z);
            body(cp.w, cz.w, ca.w);
            q = qn;
        }
    }
    for (int64_t i = e4 + tid; i < e; i += nt) body(p.pixel[i], p.z[i], p.alpha[i]);
}

// With colour: body(valid, pixel, z, alpha, r, g, b).  Trip counts are the
// same for every lane of the block (lanes past the range get valid = false),
// so the body may use warp-wide collectives.
template <class Body>
__device__ __forceinline__ void for_each_frag6(int64_t s, int64_t e, const Params &p, Body &&body) {
    const int tid = threadIdx.x, nt = blockDim.x;
    int64_t s4 = (s + 3) & ~int64_t(3), e4 = e & ~int64_t(3);
    if (s4 > e4) s4 = e4 = e;
    for (int64_t b0 = s; b0 < s4; b0 += nt) {
        const int64_t i = b0 + tid;
        const bool v = i < s4;
        body(v, v ? p.pixel[i] : 0u, v ? p.z[i] : 0.f, v ? p.alpha[i] : 0.f, v ? p.r[i] : 0.f,
             v ? p.gc[i] : 0.f, v ? p.b[i] : 0.f);
    }
    const uint4 *px4 = reinterpret_cast<const uint4 *>(p.pixel);
    const float4 *z4 = reinterpret_cast<const float4 *>(p.z);
    const float4 *a4 = reinterpret_cast<const float4 *>(p.alpha);
    const float4 *r4 = reinterpret_cast<const float4 *>(p.r);
    const float4 *g4 = reinterpret_cast<const float4 *>(p.gc);
    const float4 *b4 = reinterpret_cast<const float4 *>(p.b);
    const int64_t qe = e4 >> 2;
    {
        const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
        int64_t q = (s4 >> 2) + tid;
        bool v = q < qe;
        uint4 pv = v ? px4[q] : make_uint4(0, 0, 0, 0);
        float4 zv = v ? z4[q] : zero, av = v ? a4[q] : zero, rv = v ? r4[q] : zero;
        float4 gv = v ? g4[q] : zero, bv = v ? b4[q] : zero;
        for (int64_t q0 = s4 >> 2; q0 < qe; q0 += nt) {
            const uint4 cp = pv;
            const float4 cz = zv, ca = av, cr = rv, cg = gv, cb = bv;
            const bool cv = v;
            q += nt;
            v = q < qe;
            if (v) {  // next chunk in flight while this one is processed
                pv = px4[q];
                zv = z4[q];
                av = a4[q];
                rv = r4[q];
                gv = g4[q];
                bv = b4[q];
            }
            body(cv, cp.x, cz.x, ca.x, cr.x, cg.x, cb.x);
            body(cv, cp.y, cz.y, ca.y, cr.y, cg.y, cb.y);
            body(cv, cp.z, cz.z, ca.z, cr.z, cg.z, cb.z);
            body(cv, cp.w, cz.w, ca.w, cr.w, cg.w, cb.w);
        }
    }
    for (int64_t b0 = e4; b0 < e; b0 += nt) {
        const int64_t i = b0 + tid;
        const bool v = i < e;
        body(v, v ? p.pixel[i] : 0u, v ? p.z[i] : 0.f, v ? p.alpha[i] : 0.f, v ? p.r[i] : 0.f,
             v ? p.gc[i] : 0.f, v ? p.b[i] : 0.f);
    }
}

// ---------------------------------------------------------------- shared-memory updates

__device__ __forceinline__ void fill_zero(void *smem, int bytes) {
    float4 *p = static_cast<float4 *>(smem);
    for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Warp-segmented reduction by pixel: adds v into mine[lp] for every lane with
// lp >= 0.  Called by all 32 lanes together.  Each round, every pending lane
// writes its lane number into its pixel's byte of the warp's owner array; the
// lanes that read their own number back hold distinct pixels and update the
// warp's private accumulators with a plain read-modify-write.  Lanes that lost
// try again in the next round, so a warp needs as many rounds as its most
// repeated pixel has lanes (usually one or two) and no atomic is used.
__device__ __forceinline__ void warp_accumulate(float4 *mine, unsigned char *owner, int lp, float4 v) {
    const unsigned lane = threadIdx.x & 31;
    bool pending = lp >= 0;
    while (__any_sync(0xffffffffu, pending)) {
        if (pending) owner[lp] = (unsigned char)lane;
        __syncwarp();
        if (pending && owner[lp] == (unsigned char)lane) {
            float4 o = mine[lp];
            o.x += v.x;
            o.y += v.y;
            o.z += v.z;
            o.w += v.w;
            mine[lp] = o;
            pending = false;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- error count

__device__ __forceinline__ void flush_bad(unsigned bad, unsigned long long *err) {
    bad = __reduce_add_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(err, (unsigned long long)bad);
}

// ---------------------------------------------------------------- per-pixel transforms

// 2^{n/2} and 2^{-n/2}/2 as compile-time constants
__device__ __forceinline__ constexpr float sqrt2_pow(int n) {
    return (n & 1 ? 1.41421356237309505f : 1.f) * (float)(1u << (n >> 1));
}
__device__ __forceinline__ constexpr float half_inv_sqrt2_pow(int n) { return 0.5f / sqrt2_pow(n); }

// One level of the bins -> coefficients tree (children at level n+1 in
// F, G[0 .. 2^{n+1}), parents written to F, G[0 .. 2^n)).
template <int J, int n>
__device__ __forceinline__ void tree_level(float (&F)[1 << J], float (&G)[1 << J], float (&c)[1 << J]) {
#pragma unroll
    for (int k = 0; k < (1 << n); ++k) {
        const float t = F[2 * k] + G[2 * k + 1];
        c[(1 << n) + k] = -half_inv_sqrt2_pow(n) * t;
        const float Fp = fmaf(0.5f, t, F[2 * k + 1]);
        const float Gp = fmaf(0.5f, t, G[2 * k]);
        F[k] = Fp;
        G[k] = Gp;
    }
    if constexpr (n > 0) tree_level<J, n - 1>(F, G, c);
}

// Bins (F, G) of one pixel -> Haar coefficients in heap order, and S = sum a.
template <int J> __device__ __forceinline__ void get_row(const float *row, float (&v)[1 << J]) {
    constexpr int C = 1 << J;
    if constexpr (C % 4 == 0) {
#pragma unroll
        for (int q = 0; q < C / 4; ++q) {
            const float4 x = reinterpret_cast<const float4 *>(row)[q];
            v[4 * q] = x.x;
            v[4 * q + 1] = x.y;
            v[4 * q + 2] = x.z;
            v[4 * q + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < C; ++i) v[i] = row[i];
    }
}

template <int J>
__device__ __forceinline__ void bins_to_coeffs(const unsigned *Frow, const unsigned *Grow,
                                               float (&c)[1 << J], float &S) {
    constexpr int C = 1 << J;
    float F[C], G[C];
    const float inv = __uint_as_float(Frow[Shape<J>::INV]);  // 1 / s_p, a power of two
    get_row<J>(reinterpret_cast<const float *>(Frow), F);
    get_row<J>(reinterpret_cast<const float *>(Grow), G);
#pragma unroll
    for (int i = 0; i < C; ++i) {
        F[i] = (float)__float_as_uint(F[i]) * inv;
        G[i] = (float)__float_as_uint(G[i]) * inv;
    }
    tree_level<J, J - 1>(F, G, c);
    c[0] = G[0];
    S = F[0] + G[0];
}

// One level of the synthesis: values on the 2^n intervals of level n in
// v[0 .. 2^n) become values on the 2^{n+1} intervals of level n+1.
template <int J, int n>
__device__ __forceinline__ void synth_level(float (&v)[1 << J], const float (&c)[1 << J]) {
#pragma unroll
    for (int k = (1 << n) - 1; k >= 0; --k) {
        const float d = sqrt2_pow(n) * c[(1 << n) + k];
        const float base = v[k];
        v[2 * k + 1] = base - d;
        v[2 * k] = base + d;
    }
    if constexpr (n + 1 < J) synth_level<J, n + 1>(v, c);
}

// Haar synthesis at the bin centres, in place: values of the Haar series on
// each finest bin, A_m = chi_00 + sum_n (+-) 2^{n/2} X_{n, m >> (J-n)}.
template <int J> __device__ __forceinline__ void coeffs_to_bins(float (&v)[1 << J]) {
    float c[1 << J];
#pragma unroll
    for (int i = 0; i < (1 << J); ++i) c[i] = v[i];
    synth_level<J, 0>(v, c);
}

// Where a depth falls for the reconstruction of §2.3.2, from s = C z:
// bin m and fraction f; the interpolation segment lo (between the centres of
// bins lo and lo+1) and weight t; and g, the fragment's own unit step
// reconstructed at its own depth (its bin values are 0 before bin m, 1-f in
// it and 1 after it).  Linear: position pos = s - 1/2 in centre units,
// clamped so that the outer half-bins are constant.  Staircase: the bin value.
struct Pos {
    int m, lo;
    float f, t, g;
};
template <int J> __device__ __forceinline__ Pos locate(float s, uint32_t flags) {
    constexpr int C = 1 << J;
    Pos q;
    q.m = (int)s;
    q.f = s - (float)q.m;
    if (flags & kLinear) {
        const float pos = s - 0.5f;
        q.lo = min(max((int)floorf(pos), 0), C - 2);
        q.t = fminf(fmaxf(pos - (float)q.lo, 0.f), 1.f);
        // own bin values at lo, lo+1: (0, 1-f) when lo = m-1, (1-f, 1) when lo = m
        const float omf = 1.f - q.f;
        q.g = q.lo < q.m ? q.t * omf : fmaf(q.t, q.f, omf);
    } else {
        q.lo = q.m;
        q.t = 0.f;
        q.g = 1.f - q.f;
    }
    return q;
}

// Reconstruction at a located depth from one pixel's bin values.
template <int J>
__device__ __forceinline__ float recon_at(const float *A, const Pos &q, uint32_t flags) {
    if (!(flags & kLinear)) return A[q.m];
    const float A0 = A[q.lo], A1 = A[q.lo + 1];
    return fmaf(q.t, A1 - A0, A0);
}

// Absorbance in front of a fragment, in the units of A (a2 = its step in
// those units); the own step is removed under self-exclusion.
template <int J>
__device__ __forceinline__ float frag_absorbance(const float *A, float zc, float a2, uint32_t flags) {
    const Pos q = locate<J>(zc * (float)(1 << J), flags);
    const float full = recon_at<J>(A, q, flags);
    return (flags & kSelfExclude) ? fmaxf(full - a2 * q.g, 0.f) : full;
}

// Per-pixel weight offset m_p (log2 units): every fragment's absorbance is
// >= m_p and the nearest one's is <= m_p + 20, so 2^(m_p - A_i) never
// overflows and the largest weight never underflows.
template <int J>
__device__ __forceinline__ float weight_offset(const float *A2, float zmin, uint32_t flags) {
    if (!(zmin < 1.f)) return 0.f;  // +inf: no fragment with alpha > 0
    const float full = frag_absorbance<J>(A2, clamp_depth(zmin), 0.f, flags & kLinear);
    return fmaxf(full - kStepCapLog2, 0.f);
}

// Stores one pixel's bin values (log2 units) into its shared row and, in the
// normalised resolve, folds in the weight offset: the row becomes A' = A - m_p
// with m_p from the pixel's nearest depth (every fragment then has A' >= 0 up
// to rounding, which the self-excluded clamp at 0 absorbs).
template <int J>
__device__ __forceinline__ void put_bins(float *row, float (&v)[1 << J], float zmin, uint32_t flags) {
    constexpr int C = 1 << J;
    auto put = [&]() {
        if constexpr (C % 4 == 0) {
#pragma unroll
            for (int q = 0; q < C / 4; ++q)
                reinterpret_cast<float4 *>(row)[q] =
                    make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
#pragma unroll
            for (int i = 0; i < C; ++i) row[i] = v[i];
        }
    };
    put();
    if (!(flags & kNormalized)) return;
    const float mp = weight_offset<J>(row, zmin, flags);
    if (mp > 0.f) {
#pragma unroll
        for (int i = 0; i < C; ++i) v[i] -= mp;
        put();
    }
}

// ---------------------------------------------------------------- fragment phases

// Step 2 accumulation.  Pass 0 counts each pixel's fragments and takes its
// largest clamped alpha (integer atomics on the padding words of its F row);
// the pixel's scale s_p = 2^(30 - floor(log2(c_p a_max))) then keeps every bin
// sum below 2^32; pass 1 adds rint(s_p a f) and rint(s_p a (1-f)) to the
// fragment's bin with integer atomics, and the nearest depth with a red.min.
template <int J>
__device__ __forceinline__ void phase_bins(const Params &p, const Tile &T, unsigned *sF, unsigned *sG,
                                           unsigned *sZ, unsigned &bad) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD;
    constexpr int CNT = Shape<J>::CNT, AMAX = Shape<J>::AMAX, INV = Shape<J>::INV;
    for_each_frag2(T.s, T.e, p, [&](uint32_t px, float al) {
        if (!(al == al)) return;
        const int lp = local_pixel(px, p, T);
        if (lp < 0) return;
        atomicAdd(&sF[lp * LD + CNT], 1u);
        atomicMax(&sF[lp * LD + AMAX], __float_as_uint(clamp_alpha(al)));
    });
    __syncthreads();
    for (int lp = threadIdx.x; lp < p.g.tile_w * p.g.tile_h; lp += blockDim.x) {
        unsigned *row = sF + lp * LD;
        const float bound = (float)row[CNT] * step_of(__uint_as_float(row[AMAX]));
        const int e = bound > 0.f ? max(ilogbf(bound), -30) : 0;
        row[INV] = __float_as_uint(ldexpf(1.f, e - 30));  // 1 / s_p
        row[AMAX] = __float_as_uint(ldexpf(1.f, 30 - e));  // s_p (the maximum is no longer needed)
    }
    __syncthreads();
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
        const float sp = __uint_as_float(sF[lp * LD + AMAX]);
        const float a = step_of(clamp_alpha(al));
        const float zc = clamp_depth(z);
        const float s = zc * (float)C;  // exact: C is a power of two
        const int m = (int)s;
        const float f = s - (float)m;
        const float as = a * sp;
        atomicAdd(&sF[lp * LD + m], __float2uint_rn(as * f));
        atomicAdd(&sG[lp * LD + m], __float2uint_rn(as * (1.f - f)));
        if (a > 0.f) atomicMin(&sZ[lp], __float_as_uint(zc));
    });
}

// Step 3 (§2.1).  A2 holds each pixel's bin values in log2 units minus the
// pixel's weight offset m_p, so v_i = 2^(m_p - A_i) = 2^-A'_i and
// w_i = alpha_i v_i; per pixel (R, G, B, W) += (c w, w) through the
// warp-segmented reduction into this warp's copy, and, when sS is given,
// S += a with a shared-memory atomic.
template <int J, bool COUNT>
__device__ __forceinline__ void phase_resolve(const Params &p, const Tile &T, const float *A2,
                                              float4 *accw, unsigned char *owners, float *sS,
                                              unsigned &bad) {
    constexpr int LD = Shape<J>::LD;
    const uint32_t flags = p.flags;
    const int npx = p.g.tile_w * p.g.tile_h;
    float4 *mine = accw + (threadIdx.x >> 5) * npx;
    unsigned char *owner = owners + (threadIdx.x >> 5) * npx;
    for_each_frag6(T.s, T.e, p,
                   [&](bool valid, uint32_t px, float z, float al, float r, float g, float b) {
        int lp = -1;
        float4 c = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid) {
            if (z == z && al == al) lp = local_pixel(px, p, T);
            if (lp >= 0) {
                const float ac = clamp_alpha(al);
                const float a = step_of(ac);
                const float Ah = frag_absorbance<J>(A2 + lp * LD, clamp_depth(z), a * kLog2e, flags);
                const float w = ac * ex2(-Ah);
                c = make_float4(r * w, g * w, b * w, w);
                if (sS) atomicAdd(&sS[lp], a);
            } else if (COUNT) {
                ++bad;
            }
        }
        warp_accumulate(mine, owner, lp, c);
    });
}

// Sum over the warps' copies of pixel lp's accumulators.
__device__ __forceinline__ float4 sum_warps(const float4 *accw, int npx, int lp) {
    float4 v = accw[lp];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) {
        const float4 u = accw[w * npx + lp];
        v.x += u.x;
        v.y += u.y;
        v.z += u.z;
        v.w += u.w;
    }
    return v;
}

// ---------------------------------------------------------------- composite

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

// ---------------------------------------------------------------- shared-memory layouts (bytes)

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Every region starts on a 16-byte boundary (float4 row reads and writes).
template <int J> struct Layout {
    static constexpr size_t plane(int npx) { return align16((size_t)npx * Shape<J>::LD * 4); }
    static constexpr size_t words(int npx) { return align16((size_t)npx * 4); }
    static constexpr size_t accw(int npx) { return (size_t)kWarps * npx * 16; }
    static constexpr size_t owners(int npx) { return align16((size_t)kWarps * npx); }
    // build: F and G bins + nearest-depth words
    static constexpr size_t build(int npx) { return 2 * plane(npx) + words(npx); }
    // fused: F and G bins, replaced after the build by the bin values, the
    // warps' accumulators and the S words; then the nearest-depth words
    static constexpr size_t region(int npx) {
        return 2 * plane(npx) > plane(npx) + accw(npx) + words(npx) + owners(npx)
                   ? 2 * plane(npx)
                   : plane(npx) + accw(npx) + words(npx) + owners(npx);
    }
    static constexpr size_t fused(int npx) { return region(npx) + words(npx); }
    // resolve: bin values + warps' accumulators + S words + owner bytes
    static constexpr size_t resolve(int npx) { return plane(npx) + accw(npx) + words(npx) + owners(npx); }
};

}  // namespace wt
