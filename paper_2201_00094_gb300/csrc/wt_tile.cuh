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
// The bins are 32-bit fixed point (scale 2^27; a tile whose bins would wrap is
// rebuilt with per-pixel scales from a counting pass) and are added with
// integer atomics: the sums do not depend on the order of the fragments, so
// the coefficients -- and everything computed from them in one CTA -- are the
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
// The build's F and G bins live in separate shared planes, so a warp's lanes
// spread over the banks.  The resolve's per-pixel sums use a warp-segmented
// reduction instead of atomics: the lanes of a warp that hold the same pixel
// are ranked (match.any) and update the warp's private copy of the
// accumulators in rank order with plain read-modify-writes; the copies are
// summed per pixel at the end of the tile.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace wt {

constexpr int kThreads = 256;    // threads per CTA (= max pixels per tile)
constexpr int kMaxTilePx = 256;
constexpr int kWarps = kThreads / 32;  // warp-private copies of the per-pixel accumulators
// alpha is clamped to [0, 1 - 2^-20] and z to [0, 1 - 2^-24] (exact in FP32)
constexpr float kAlphaMax = 0.99999904632568359375f;
constexpr float kZMax = 0.999999940395355224609375f;
constexpr float kLog2e = 1.44269504088896340736f;
// the largest step after the clamp is -ln(2^-20) = 20 ln 2, i.e. 20 in log2 units
constexpr float kStepCapLog2 = 20.0f;

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

struct Geom {
    int width, height, tile_w, tile_h, ntx;
};

// Everything a kernel reads or writes; passed by value.
struct Params {
    Geom g;
    int32_t tile0;  // first tile of a fused launch (block b works on tile tile0 + b)
    uint32_t flags;
    uint32_t wmagic32;  // ceil(2^32 / width) when that divides every in-tile offset exactly, else 0
    uint64_t wmagic;    // ceil(2^64 / width) (0 when width == 1)
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
    float *total;  // per-pixel total step S: written by the build, read by the resolve (nullable)
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
// the default method: self-excluded, linearly interpolated, normalised resolve
constexpr uint32_t kDefaultFlags = kSelfExclude | kLinear | kNormalized;

template <int J> struct Shape {
    static constexpr int C = 1 << J;
    static constexpr int LD = C + 4;  // words per pixel row of bins (16-byte rows)
    // the padding words of a pixel's F row hold its counting-pass results
    static constexpr int CNT = C, AMAX = C + 1, INV = C + 2;
    // Row of bin values: word V0 + m holds A_m, and the row is padded on both
    // sides with copies of the end values (word V0 - 1 = A_0, word V0 + C =
    // A_{C-1}), so the linear reconstruction reads entries lo, lo + 1 of the
    // padded sequence at words V0 - 1 + lo for every lo in [0, C] with no
    // clamping.  The row length is odd, so that rows start on 32 different
    // banks: the lanes of a warp read random pixels' rows, often at the same
    // bin (fragments cluster in depth), and a stride of C + 8 words put rows
    // four apart on the same bank (1.7% of the fused kernel's time at 4K).
    static constexpr int V0 = 1, LDV = C + 3;
};

// The build's bins are 32-bit fixed point, F and G scaled by 2^27: one
// fragment adds at most 20 ln 2 * 2^27 < 2^31, and a bin holds up to 32
// absorbance units before its word wraps.  A wrap is detected from the atomic's
// return value; the tile is then rebuilt with per-pixel scales (a counting pass
// bounds every pixel's sums), so the bins never overflow.  Tiles holding a step
// below 2^-7 are rebuilt the same way, so every step keeps a relative
// resolution of 2^-21 or better.
constexpr float kBinScale = 134217728.f;              // 2^27
constexpr float kBinInv = 7.450580596923828125e-9f;  // 2^-27

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

// E5B9G9R9: three non-negative values with one shared 5-bit exponent (bias
// 15) and 9-bit mantissas, the 32-bit coefficient format of the paper's
// coloured storage (its coefficients have fixed signs, §2.3.1, so magnitudes
// suffice).  Encoding follows the published shared-exponent format: clamp to
// the largest representable value, take the exponent from the largest channel
// (one more if its rounded mantissa reaches 2^9), round every mantissa to
// nearest.
constexpr float kE5Max = 65408.f;  // (511/512) * 2^16
// 2^k for -126 <= k <= 127
__device__ __forceinline__ float exp2i(int k) { return __int_as_float((127 + k) << 23); }
// The shared exponent of three clamped values whose largest is mx, with
// scale = 2^(24 - e) (value -> mantissa units) and unit = 2^(e - 24).
struct E5Scale {
    int e;
    float scale, unit;
};
__device__ __forceinline__ float e5_clamp(float x) { return fminf(fmaxf(x, 0.f), kE5Max); }  // NaN -> 0
// floor(x scale + 1/2) for x scale + 1/2 < 2^23: the fma rounds once, and the
// round-toward-zero add of 2^23 leaves the floor in the low mantissa bits
__device__ __forceinline__ uint32_t e5_mant(float x, float scale) {
    return (uint32_t)(__float_as_int(__fadd_rz(fmaf(x, scale, 0.5f), 8388608.f)) - 0x4B000000);
}
__device__ __forceinline__ E5Scale e5_scale(float mx) {
    // floor(log2(mx)) for mx > 0, from the exponent bits (subnormal FP32 values
    // are far below the format's smallest exponent and take the floor -16)
    const int fl = mx > 0.f ? max(((int)(__float_as_uint(mx) >> 23) & 0xff) - 127, -16) : -16;
    E5Scale s;
    s.e = fl + 1 + 15;  // in [0, 32)
    s.scale = exp2i(24 - s.e);
    if (e5_mant(mx, s.scale) >= 512u) {
        ++s.e;
        s.scale *= 0.5f;
    }
    s.unit = exp2i(s.e - 24);
    return s;
}
__device__ __forceinline__ uint32_t e5_encode(float r, float g, float b) {
    r = e5_clamp(r);
    g = e5_clamp(g);
    b = e5_clamp(b);
    const E5Scale s = e5_scale(fmaxf(r, fmaxf(g, b)));
    return e5_mant(r, s.scale) | (e5_mant(g, s.scale) << 9) | (e5_mant(b, s.scale) << 18) | ((uint32_t)s.e << 27);
}
__device__ __forceinline__ void e5_decode(uint32_t w, float &r, float &g, float &b) {
    const float unit = exp2i((int)(w >> 27) - 24);
    r = (float)(w & 511u) * unit;
    g = (float)((w >> 9) & 511u) * unit;
    b = (float)((w >> 18) & 511u) * unit;
}

// Shared-exponent 16-bit storage (WT_SE16).  The sign property of §2.3.1
// (chi_00 >= 0, every X_{n,k} <= 0) makes every coefficient a magnitude, as in
// the paper's E5B9G9R9 words (§2.1); here one exponent is shared by the 2^J
// coefficients of a pixel.  Per pixel: m_0 = chi_00 and m_i = -X_{n,k}
// 2^floor(n/2) (i = 2^n + k), so that every m_i is at most the pixel's total
// step; e = floor(log2 max m) + 1 (clamped to [-100, 100]), q_i =
// rint(m_i 2^(16 - e)) as unsigned 16-bit mantissas, e raised by one when the
// largest q reaches 2^16.  The mantissas sit where a 16-bit row would,
// [P][C] pixel-major; the P exponent bytes (e + 128) follow them.  Every
// decoded value is q_i 2^(e - 16 - floor(n/2)) exactly, and its error is at
// most half a unit of the pixel's largest magnitude, not of its own size.
struct se16_t {
    uint16_t q;
};
template <typename CT> constexpr bool kIsSE16 = std::is_same<CT, se16_t>::value;
constexpr int kSE16Emin = -100, kSE16Emax = 100, kSE16Bias = 128;

// 2^floor(n/2) for heap index i = 2^n + k (1 for chi_00); constant-folded in
// unrolled loops
__device__ __forceinline__ float se16_level_scale(int i) {
    return i > 0 ? (float)(1 << ((31 - __clz(i)) >> 1)) : 1.f;
}
// q as a float for q < 2^23 (2^23 + q is exact; subtracting 2^23 leaves q)
__device__ __forceinline__ float small_to_float(uint32_t q) { return __uint_as_float(0x4B000000u | q) - 8388608.f; }

// Byte plane of the exponents behind the P * C mantissas.
template <int C> __device__ __forceinline__ uint8_t *se16_expo(const void *coeff, int64_t P) {
    return (uint8_t *)coeff + (size_t)P * C * 2;
}

// Encodes a row in place: v becomes the decoded values; returns e.  The
// coefficients come from the bins tree (or sums of its rows), which gives
// chi_00 >= 0 and X_{n,k} <= 0, so |v_i| is the clamped magnitude of the
// definition.  Rounding: m 2^(16-e) + 2^23 (one FMA, exact product) rounds
// half to even onto the integers 2^23 + q; decoding subtracts 2^23 and scales
// (one more FMA), which is exact.
template <int C> __device__ __forceinline__ int se16_round(float (&v)[C]) {
    float m[C];
    float M = 0.f;
#pragma unroll
    for (int i = 0; i < C; ++i) {
        m[i] = fabsf(v[i]) * se16_level_scale(i);
        M = fmaxf(M, m[i]);
    }
    const int ex = (__float_as_int(M) >> 23) & 0xff;
    int e = ex > 0 ? min(max(ex - 126, kSE16Emin), kSE16Emax) : kSE16Emin;
    float scale = exp2i(16 - e);
    if (fmaf(M, scale, 8388608.f) >= 8388608.f + 65536.f) {  // the largest q reached 2^16
        ++e;
        scale *= 0.5f;
    }
    const float unit = exp2i(e - 16);
#pragma unroll
    for (int i = 0; i < C; ++i) {
        const float r = fmaf(m[i], scale, 8388608.f);  // 2^23 + q_i
        const float c = (i == 0 ? unit : -unit) / se16_level_scale(i);
        v[i] = fmaf(r, c, -8388608.f * c);  // (r - 2^23) c, exact
    }
    return e;
}

// Rounds a row to the storage precision in place (the values the resolve
// uses) and returns the row's shared exponent (0 for the per-element types).
template <typename CT, int C> __device__ __forceinline__ int round_row(float (&v)[C]) {
    if constexpr (kIsSE16<CT>) {
        return se16_round<C>(v);
    } else {
#pragma unroll
        for (int i = 0; i < C; ++i) v[i] = Cvt<CT>::from(Cvt<CT>::to(v[i]));
        return 0;
    }
}
// The shared exponent of a row about to be stored; rounds the row in place
// for WT_SE16 and leaves the per-element types untouched (their stores round).
template <typename CT, int C> __device__ __forceinline__ int storage_exponent(float (&v)[C]) {
    if constexpr (kIsSE16<CT>) return se16_round<C>(v);
    else return 0;
}

// Element i of a row to / from storage form.  For WT_SE16, v must already be
// a decoded value of the row (round_row / storage_exponent) and scale =
// 2^(16 - e), unit = 2^(e - 16) for the row's exponent e; the mantissa is then
// exact.
template <typename CT> __device__ __forceinline__ CT to_storage(float v, int i, float scale) {
    if constexpr (kIsSE16<CT>)
        return CT{(uint16_t)(__float_as_int(fmaf(fabsf(v), scale * se16_level_scale(i), 8388608.f)) - 0x4B000000)};
    else return Cvt<CT>::to(v);
}
template <typename CT> __device__ __forceinline__ float from_storage(CT x, int i, float unit) {
    if constexpr (kIsSE16<CT>) {
        const float d = small_to_float(x.q) * (unit / se16_level_scale(i));
        return i == 0 ? d : -d;
    } else {
        return Cvt<CT>::from(x);
    }
}
__device__ __forceinline__ float se16_scale(int e) { return exp2i(16 - e); }
__device__ __forceinline__ float se16_unit(int e) { return exp2i(e - 16); }

// One pixel's C coefficients to / from global memory, 16-byte vectors when
// the row is a multiple of 16 bytes (it is 16-byte aligned then).  e is the
// row's shared exponent (WT_SE16; ignored otherwise).
template <typename CT, int C>
__device__ __forceinline__ void store_row(CT *dst, const float (&v)[C], int e = 0) {
    constexpr int PER = 16 / sizeof(CT);
    const float scale = kIsSE16<CT> ? se16_scale(e) : 0.f;
    if constexpr (C % PER == 0) {
#pragma unroll
        for (int q = 0; q < C / PER; ++q) {
            union { uint4 u; CT x[PER]; } pk;
#pragma unroll
            for (int i = 0; i < PER; ++i) pk.x[i] = to_storage<CT>(v[q * PER + i], q * PER + i, scale);
            reinterpret_cast<uint4 *>(dst)[q] = pk.u;
        }
    } else {
#pragma unroll
        for (int i = 0; i < C; ++i) dst[i] = to_storage<CT>(v[i], i, scale);
    }
}

template <typename CT, int C>
__device__ __forceinline__ void load_row(const CT *src, float (&v)[C], int e = 0) {
    constexpr int PER = 16 / sizeof(CT);
    const float unit = kIsSE16<CT> ? se16_unit(e) : 0.f;
    if constexpr (C % PER == 0) {
#pragma unroll
        for (int q = 0; q < C / PER; ++q) {
            union { uint4 u; CT x[PER]; } pk;
            pk.u = reinterpret_cast<const uint4 *>(src)[q];
#pragma unroll
            for (int i = 0; i < PER; ++i) v[q * PER + i] = from_storage<CT>(pk.x[i], q * PER + i, unit);
        }
    } else {
#pragma unroll
        for (int i = 0; i < C; ++i) v[i] = from_storage<CT>(src[i], i, unit);
    }
}

// Coefficient rows of a tile staged in shared memory, so that they reach
// global memory in coalesced 16-byte vectors (a thread's own 128-byte row
// written directly would touch 32 cache lines per warp instruction).  A row of
// K = C * sizeof(CT) / 16 chunks is staged at chunks lp*K .. lp*K + K-1 with
// chunk q at position q ^ sw(lp): the eight lanes of a quarter warp then
// write eight distinct bank groups.
template <typename CT, int C> struct Staged {
    static constexpr bool ok = (C * (int)sizeof(CT)) % 16 == 0;
    static constexpr int K = ok ? C * (int)sizeof(CT) / 16 : 1;  // (unused when not ok)
    static __device__ __forceinline__ int sw(int lp) { return (lp / (K >= 8 ? 1 : 8 / K)) & (K - 1); }
};

template <typename CT, int C>
__device__ __forceinline__ void stage_row(uint4 *stage, int lp, const float (&v)[C], int e = 0) {
    using S = Staged<CT, C>;
    constexpr int PER = 16 / sizeof(CT);
    const int sw = S::sw(lp);
    const float scale = kIsSE16<CT> ? se16_scale(e) : 0.f;
#pragma unroll
    for (int q = 0; q < S::K; ++q) {
        union { uint4 u; CT x[PER]; } pk;
#pragma unroll
        for (int i = 0; i < PER; ++i) pk.x[i] = to_storage<CT>(v[q * PER + i], q * PER + i, scale);
        stage[lp * S::K + (q ^ sw)] = pk.u;
    }
}

template <typename CT, int C>
__device__ __forceinline__ void unstage_row(const uint4 *stage, int lp, float (&v)[C], int e = 0) {
    using S = Staged<CT, C>;
    constexpr int PER = 16 / sizeof(CT);
    const int sw = S::sw(lp);
    const float unit = kIsSE16<CT> ? se16_unit(e) : 0.f;
#pragma unroll
    for (int q = 0; q < S::K; ++q) {
        union { uint4 u; CT x[PER]; } pk;
        pk.u = stage[lp * S::K + (q ^ sw)];
#pragma unroll
        for (int i = 0; i < PER; ++i) v[q * PER + i] = from_storage<CT>(pk.x[i], q * PER + i, unit);
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
// d = pixel - tile origin.  A tile one row high (a span of a row) needs no
// division.  Otherwise the row is d / width, taken as the high word of
// d * ceil(2^32 / width) when the host has shown that exact for every
// d < tile_h * width, else of d * ceil(2^64 / width), exact for any 32-bit d
// (Granlund & Montgomery 1994).
__device__ __forceinline__ int local_pixel(uint32_t px, const Params &p, const Tile &T) {
    const uint32_t d = px - T.base;
    if (p.g.tile_h == 1) return d < (uint32_t)T.tw ? (int)d : -1;
    if (d >= T.lim) return -1;
    const uint32_t ly = p.wmagic32 ? __umulhi(d, p.wmagic32)
                                   : (p.wmagic ? (uint32_t)__umul64hi((uint64_t)d, p.wmagic) : d);
    const uint32_t lx = d - ly * (uint32_t)p.g.width;
    if (lx >= (uint32_t)T.tw) return -1;
    return (int)(ly * (uint32_t)p.g.tile_w + lx);
}

// Host side: the two magic numbers of the row division for width and tile_h.
// With m = ceil(2^32 / w) = (2^32 + e) / w, floor(d m / 2^32) = floor(d / w)
// whenever d e < 2^32, so the 32-bit form is used when (tile_h w - 1) e < 2^32.
inline void set_row_division(Params &p) {
    const unsigned long long w = (unsigned long long)p.g.width;
    p.wmagic = w > 1 ? ~0ull / w + 1ull : 0ull;
    p.wmagic32 = 0;
    if (w > 1) {
        const unsigned long long m = ((1ull << 32) + w - 1) / w;
        const unsigned long long e = m * w - (1ull << 32);
        const unsigned long long dmax = (unsigned long long)p.g.tile_h * w - 1;
        if (m < (1ull << 32) && dmax * e < (1ull << 32)) p.wmagic32 = (uint32_t)m;
    }
}

// global pixel id of local pixel lp, or -1 if it lies outside the image
__device__ __forceinline__ int64_t global_pixel(const Params &p, const Tile &T, int lp) {
    const int lx = lp % p.g.tile_w, ly = lp / p.g.tile_w;
    if (lx >= T.tw || ly >= T.th) return -1;
    return (int64_t)(T.ty0 + ly) * p.g.width + T.tx0 + lx;
}

// Copies the staged coefficient rows of a tile to global memory (consecutive
// threads take consecutive 16-byte chunks: a tile row's pixels are contiguous
// in the pixel-major coefficient array) and clears the staging area, whose
// `bytes` bytes are reused as zeroed accumulators afterwards.
template <typename CT, int C>
__device__ __forceinline__ void copy_staged(const Params &p, const Tile &T, uint4 *stage, int bytes,
                                            CT *coeff) {
    using S = Staged<CT, C>;
    const int npx = p.g.tile_w * p.g.tile_h;
    const int nchunk = npx * S::K;
    for (int c = threadIdx.x; c < bytes / 16; c += blockDim.x) {
        if (c < nchunk) {
            const int lp = c / S::K, q = (c % S::K) ^ S::sw(lp);
            int lx = lp, ly = 0;
            if (p.g.tile_h != 1) {
                lx = lp % p.g.tile_w;
                ly = lp / p.g.tile_w;
            }
            if (lx < T.tw && ly < T.th) {
                const int64_t gp = (int64_t)(T.ty0 + ly) * p.g.width + T.tx0 + lx;
                reinterpret_cast<uint4 *>(coeff + gp * C)[q] = stage[c];
            }
        }
        stage[c] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// The reverse of copy_staged: a tile's coefficient rows read from global
// memory in coalesced 16-byte chunks into their staged positions.
template <typename CT, int C>
__device__ __forceinline__ void load_staged(const Params &p, const Tile &T, uint4 *stage,
                                            const CT *coeff) {
    using S = Staged<CT, C>;
    const int nchunk = p.g.tile_w * p.g.tile_h * S::K;
    for (int c = threadIdx.x; c < nchunk; c += blockDim.x) {
        const int lp = c / S::K, q = (c % S::K) ^ S::sw(lp);
        int lx = lp, ly = 0;
        if (p.g.tile_h != 1) {
            lx = lp % p.g.tile_w;
            ly = lp / p.g.tile_w;
        }
        if (lx < T.tw && ly < T.th) {
            const int64_t gp = (int64_t)(T.ty0 + ly) * p.g.width + T.tx0 + lx;
            stage[c] = reinterpret_cast<const uint4 *>(coeff + gp * C)[q];
        }
    }
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

// floor(x) for 0 <= x < 2^23, as an integer and as a float, on the FP32 adder
// instead of the conversion unit: x + 2^23 rounded toward zero is exactly
// 2^23 + floor(x) (the representable numbers in [2^23, 2^24) are the
// integers), whose low mantissa bits are floor(x).
struct Floor {
    int i;
    float f;
};
__device__ __forceinline__ Floor floor_small(float x) {
    const float big = __fadd_rz(x, 8388608.f);
    return {__float_as_int(big) - 0x4B000000, big - 8388608.f};
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

// Up to four consecutive fragments held by one thread.  Only the arrays a
// phase asks for are loaded (the others stay unset and are optimised away);
// kWithR loads the r array alone (one colour component).
enum : int { kWithZ = 1, kWithRGB = 2, kWithR = 4 };
template <int N> struct Group {
    static constexpr int size = N;
    bool v;      // inside the range (all N fragments or none)
    int64_t i0;  // index of the first fragment
    uint32_t px[N];
    float al[N], z[N], r[N], g[N], b[N];
};

template <int LOAD>
__device__ __forceinline__ void load_one(Group<1> &G, bool v, int64_t i, const Params &p) {
    G.v = v;
    G.i0 = i;
    G.px[0] = v ? p.pixel[i] : 0u;
    G.al[0] = v ? p.alpha[i] : 0.f;
    if (LOAD & kWithZ) G.z[0] = v ? p.z[i] : 0.f;
    if (LOAD & kWithRGB) {
        G.r[0] = v ? p.r[i] : 0.f;
        G.g[0] = v ? p.gc[i] : 0.f;
        G.b[0] = v ? p.b[i] : 0.f;
    }
    if (LOAD & kWithR) G.r[0] = v ? p.r[i] : 0.f;
}

template <int LOAD>
__device__ __forceinline__ void load_four(Group<4> &G, bool v, int64_t q, const Params &p) {
    uint4 pv = make_uint4(0u, 0u, 0u, 0u);
    float4 av = make_float4(0.f, 0.f, 0.f, 0.f), zv = av, rv = av, gv = av, bv = av;
    if (v) {
        pv = reinterpret_cast<const uint4 *>(p.pixel)[q];
        av = reinterpret_cast<const float4 *>(p.alpha)[q];
        if (LOAD & kWithZ) zv = reinterpret_cast<const float4 *>(p.z)[q];
        if (LOAD & kWithRGB) {
            rv = reinterpret_cast<const float4 *>(p.r)[q];
            gv = reinterpret_cast<const float4 *>(p.gc)[q];
            bv = reinterpret_cast<const float4 *>(p.b)[q];
        }
        if (LOAD & kWithR) rv = reinterpret_cast<const float4 *>(p.r)[q];
    }
    G.v = v;
    G.i0 = 4 * q;
    G.px[0] = pv.x, G.px[1] = pv.y, G.px[2] = pv.z, G.px[3] = pv.w;
    G.al[0] = av.x, G.al[1] = av.y, G.al[2] = av.z, G.al[3] = av.w;
    G.z[0] = zv.x, G.z[1] = zv.y, G.z[2] = zv.z, G.z[3] = zv.w;
    G.r[0] = rv.x, G.r[1] = rv.y, G.r[2] = rv.z, G.r[3] = rv.w;
    G.g[0] = gv.x, G.g[1] = gv.y, G.g[2] = gv.z, G.g[3] = gv.w;
    G.b[0] = bv.x, G.b[1] = bv.y, G.b[2] = bv.z, G.b[3] = bv.w;
}

// Calls body(Group<4>) for the 16-byte-aligned middle of the fragment range
// [s, e) -- one vector load per array, the next group's loads in flight while
// the body runs -- and body(Group<1>) once, in the
// block's last warp, for the unaligned head and tail (at most 3 + 3
// fragments).  Every lane of a warp makes the same calls (lanes past the range
// get v = false) and a warp stops as soon as its first lane is past the range,
// so the body may use warp-wide collectives but no block-wide barrier.  A body
// that finishes all of a group's arithmetic before its shared-memory updates
// lets the four fragments' latencies overlap.
template <int LOAD, class Body>
__device__ __forceinline__ void for_each_group(int64_t s, int64_t e, const Params &p, Body &&body) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    int64_t s4 = (s + 3) & ~int64_t(3), e4 = e & ~int64_t(3);
    if (s4 > e4) s4 = e4 = e;
    const int nh = (int)(s4 - s), ne = nh + (int)(e - e4);
    if (ne > 0 && (tid >> 5) == (nt >> 5) - 1) {
        Group<1> G;
        load_one<LOAD>(G, lane < ne, lane < nh ? s + lane : e4 + (lane - nh), p);
        body(G);
    }
    const int64_t qe = e4 >> 2;
    int64_t q = (s4 >> 2) + tid;  // the warp's first lane is at q - lane
    Group<4> next;
    load_four<LOAD>(next, q < qe, q, p);
    while (q - lane < qe) {
        Group<4> cur = next;
        q += nt;
        load_four<LOAD>(next, q < qe, q, p);
        body(cur);
    }
}

// L2 prefetch (bulk, asynchronous) of the 16-byte-aligned interior of the
// byte range [a + lo, a + hi), in pieces of at most 32 KB: a block's input
// streams into L2 while the block works on it, instead of arriving one
// register group at a time.  The bulk copy wants 16-byte aligned addresses
// and sizes, so the bounds are rounded inwards on the addresses themselves
// (any base alignment); addresses stay inside the range.
__device__ __forceinline__ void l2_prefetch_bytes(const void *a, int64_t lo, int64_t hi) {
    const uintptr_t base = reinterpret_cast<uintptr_t>(a);
    const uintptr_t p0 = (base + (uintptr_t)lo + 15) & ~uintptr_t(15), p1 = (base + (uintptr_t)hi) & ~uintptr_t(15);
    for (uintptr_t q = p0; q < p1; q += 32768) {
        const unsigned n = (unsigned)(p1 - q < 32768 ? p1 - q : 32768);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q), "r"(n) : "memory");
    }
}
// The same for the 4-byte-element range a[s, e).
__device__ __forceinline__ void l2_prefetch_range(const void *a, int64_t s, int64_t e) {
    l2_prefetch_bytes(a, s * 4, e * 4);
}
template <int LOAD> __device__ __forceinline__ void prefetch_tile(const Params &p, const Tile &T) {
    if (threadIdx.x != 0) return;
    l2_prefetch_range(p.pixel, T.s, T.e);
    l2_prefetch_range(p.alpha, T.s, T.e);
    if (LOAD & kWithZ) l2_prefetch_range(p.z, T.s, T.e);
    if (LOAD & kWithRGB) {
        l2_prefetch_range(p.r, T.s, T.e);
        l2_prefetch_range(p.gc, T.s, T.e);
        l2_prefetch_range(p.b, T.s, T.e);
    }
}

// Stores a group's N per-fragment results at dst[i0 ..], as one 16-byte
// vector when N = 4 and the address allows it.
template <int N> __device__ __forceinline__ void store_group(float *dst, int64_t i0, const float (&v)[N]) {
    if constexpr (N == 4) {
        if ((reinterpret_cast<uintptr_t>(dst + i0) & 15) == 0) {
            *reinterpret_cast<float4 *>(dst + i0) = make_float4(v[0], v[1], v[2], v[3]);
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < N; ++k) dst[i0 + k] = v[k];
}

// Loads N per-fragment values src[i0 ..] (zeros when v is false), as one
// 16-byte vector when N = 4 and the address allows it.
template <int N>
__device__ __forceinline__ void load_group(const float *src, int64_t i0, bool v, float (&x)[N]) {
#pragma unroll
    for (int k = 0; k < N; ++k) x[k] = 0.f;
    if (!v) return;
    if constexpr (N == 4) {
        if ((reinterpret_cast<uintptr_t>(src + i0) & 15) == 0) {
            const float4 q = *reinterpret_cast<const float4 *>(src + i0);
            x[0] = q.x, x[1] = q.y, x[2] = q.z, x[3] = q.w;
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < N; ++k) x[k] = src[i0 + k];
}

// ---------------------------------------------------------------- shared-memory updates

__device__ __forceinline__ void fill_zero(void *smem, int bytes) {
    float4 *p = static_cast<float4 *>(smem);
    for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// Warp-segmented reduction by pixel: adds v into mine[lp] for every lane with
// lp >= 0.  Called by all 32 lanes together.  The lanes holding the same pixel
// are grouped (match.any) and ranked by lane number; in round r the lanes of
// rank r -- at most one per pixel -- update the warp's private accumulators
// with a plain read-modify-write.  A warp needs as many rounds as its most
// repeated pixel has lanes (usually one or two), and no atomic is used.  The
// order of the additions depends only on the lanes' contents, so the sums are
// the same on every run.
__device__ __forceinline__ void accumulate_into(float4 *mine, int lp, float4 v) {
    float4 o = mine[lp];
    o.x += v.x;
    o.y += v.y;
    o.z += v.z;
    o.w += v.w;
    mine[lp] = o;
}
__device__ __forceinline__ void warp_accumulate(float4 *mine, int lp, float4 v) {
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    const unsigned rank = __popc(__match_any_sync(0xffffffffu, lp) & lt);
    if (lp >= 0 && rank == 0) accumulate_into(mine, lp, v);
    __syncwarp();
    for (unsigned r = 1; __any_sync(0xffffffffu, lp >= 0 && rank >= r); ++r) {
        if (lp >= 0 && rank == r) accumulate_into(mine, lp, v);
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
__device__ __forceinline__ void tree_level(float (&F)[1 << J], float (&G)[1 << J], float (&c)[1 << J],
                                           float inv) {
    const float h = -half_inv_sqrt2_pow(n) * inv;
#pragma unroll
    for (int k = 0; k < (1 << n); ++k) {
        const float t = F[2 * k] + G[2 * k + 1];
        c[(1 << n) + k] = h * t;
        const float Fp = fmaf(0.5f, t, F[2 * k + 1]);
        const float Gp = fmaf(0.5f, t, G[2 * k]);
        F[k] = Fp;
        G[k] = Gp;
    }
    if constexpr (n > 0) tree_level<J, n - 1>(F, G, c, inv);
}

// Bins (F, G) of one pixel -> Haar coefficients in heap order, and S = sum a.
template <int J> __device__ __forceinline__ void get_row(const float *row, float (&v)[1 << J]) {
    constexpr int C = 1 << J;
    if constexpr (C % 4 == 0 && Shape<J>::LD % 4 == 0) {  // 16-byte rows
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
__device__ __forceinline__ void bins_to_coeffs_inv(const unsigned *Frow, const unsigned *Grow, float inv,
                                                   float (&c)[1 << J], float &S);
template <int J>
__device__ __forceinline__ void bins_to_coeffs(const unsigned *Frow, const unsigned *Grow,
                                               float (&c)[1 << J], float &S, bool scaled) {
    // 1 / s_p (a power of two) when the tile took per-pixel scales, else 2^-27
    bins_to_coeffs_inv<J>(Frow, Grow, scaled ? __uint_as_float(Frow[Shape<J>::INV]) : kBinInv, c, S);
}
// The same with the fixed-point scale's reciprocal given.
template <int J>
__device__ __forceinline__ void bins_to_coeffs_inv(const unsigned *Frow, const unsigned *Grow, float inv,
                                                   float (&c)[1 << J], float &S) {
    constexpr int C = 1 << J;
    float F[C], G[C];
    get_row<J>(reinterpret_cast<const float *>(Frow), F);
    get_row<J>(reinterpret_cast<const float *>(Grow), G);
    // the tree runs on the integer sums (exact as floats up to 2^24, rounded
    // once above) and the scale enters through the level constants
#pragma unroll
    for (int i = 0; i < C; ++i) {
        F[i] = (float)__float_as_uint(F[i]);
        G[i] = (float)__float_as_uint(G[i]);
    }
    tree_level<J, J - 1>(F, G, c, inv);
    c[0] = G[0] * inv;
    S = (F[0] + G[0]) * inv;
}

// One level of the synthesis: values on the 2^n intervals of level n in
// v[0 .. 2^n) become values on the 2^{n+1} intervals of level n+1.
template <int J, int n>
__device__ __forceinline__ void synth_level(float (&v)[1 << J], const float (&c)[1 << J], float scale) {
#pragma unroll
    for (int k = (1 << n) - 1; k >= 0; --k) {
        const float d = (sqrt2_pow(n) * scale) * c[(1 << n) + k];
        const float base = v[k];
        v[2 * k + 1] = base - d;
        v[2 * k] = base + d;
    }
    if constexpr (n + 1 < J) synth_level<J, n + 1>(v, c, scale);
}

// Haar synthesis at the bin centres, in place: values of the Haar series on
// each finest bin, A_m = chi_00 + sum_n (+-) 2^{n/2} X_{n, m >> (J-n)},
// multiplied by scale (a constant folded into the level factors).
template <int J> __device__ __forceinline__ void coeffs_to_bins(float (&v)[1 << J], float scale = 1.f) {
    float c[1 << J];
#pragma unroll
    for (int i = 0; i < (1 << J); ++i) c[i] = v[i];
    v[0] = c[0] * scale;
    if constexpr (J > 0) synth_level<J, 0>(v, c, scale);
}

// Where a depth falls for the reconstruction of §2.3.2, from s = C z:
// bin m and fraction f; the interpolation segment lo (between the centres of
// bins lo and lo+1) and weight t; and g, the fragment's own unit step
// reconstructed at its own depth (its bin values are 0 before bin m, 1-f in
// it and 1 after it).  Linear: position pos = s - 1/2 in centre units,
// clamped so that the outer half-bins are constant.  Staircase: the bin value.
// (The adjoint uses every field; the forward resolve uses absorbance_at.)
struct Pos {
    int m, lo;
    float f, t, g;
};
template <int J> __device__ __forceinline__ Pos locate(float s, uint32_t flags) {
    constexpr int C = 1 << J;
    Pos q;
    const Floor fm = floor_small(s);
    q.m = fm.i;
    q.f = s - fm.f;
    if (flags & kLinear) {
        // pos clamped to [0, C-1]: lo = min(floor(pos), C-2), t = pos - lo,
        // which is t = 0 left of the first centre and t = 1 right of the last
        const float pos = fminf(fmaxf(s - 0.5f, 0.f), (float)(C - 1));
        const Floor fl = floor_small(pos);
        q.lo = min(fl.i, C - 2);
        q.t = pos - fminf(fl.f, (float)(C - 2));
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

// Reconstruction at a located depth from one pixel's row of bin values.
template <int J>
__device__ __forceinline__ float recon_at(const float *row, const Pos &q, uint32_t flags) {
    const float *A = row + Shape<J>::V0;
    if (!(flags & kLinear)) return A[q.m];
    const float A0 = A[q.lo], A1 = A[q.lo + 1];
    return fmaf(q.t, A1 - A0, A0);
}

// Absorbance in front of a fragment at clamped depth zc from its pixel's row
// of bin values, in the row's units; a2 is the fragment's own step in those
// units, removed under self-exclusion (pass 0 for the reconstruction alone).
//
// Linear interpolation: with s = C zc, the bin boundary nearest to s is
// lo = floor(s + 1/2) in [0, C] and u = s - lo in [-1/2, 1/2) is the signed
// distance to it.  The reconstruction runs between the centres on either side
// of that boundary -- entries lo, lo+1 of the padded row, weight t = u + 1/2 --
// and is constant in the outer half-bins, where both entries hold the end value.
// The own unit step reconstructed at its own depth (bin values 0, 1-f, 1 before,
// in and after its bin m, f = s - m) is then
//     g = 1/2 + u (1/2 - |u|)                  between the outer half-bins,
//     g = 1 - u  (lo = 0),   g = -u  (lo = C)  in the first / last half-bin,
// i.e. (1-f)(f+1/2) for f < 1/2 and 1 - 3f/2 + f^2 for f >= 1/2 inside.
// Staircase: the value of bin m, own step 1 - f.
template <int J>
__device__ __forceinline__ float absorbance_at(const float *row, float zc, float a2, uint32_t flags) {
    constexpr int C = 1 << J;
    const float s = zc * (float)C;  // exact: C is a power of two
    float A, g;
    if (flags & kLinear) {
        const Floor b = floor_small(s + 0.5f);
        const float u = s - b.f;  // exact
        const float *e = row + (Shape<J>::V0 - 1) + b.i;
        const float A0 = e[0], A1 = e[1];
        A = fmaf(u + 0.5f, A1 - A0, A0);
        const float inner = fmaf(u, 0.5f - fabsf(u), 0.5f);
        const float outer = (b.i == 0 ? 1.f : 0.f) - u;
        g = (unsigned)(b.i - 1) < (unsigned)(C - 1) ? inner : outer;
    } else {
        const Floor m = floor_small(s);
        A = row[Shape<J>::V0 + m.i];
        g = 1.f - (s - m.f);
    }
    return (flags & kSelfExclude) ? fmaxf(fmaf(-a2, g, A), 0.f) : A;
}

// Per-pixel weight offset m_p (log2 units): every fragment's absorbance is
// >= m_p and the nearest one's is <= m_p + 20, so 2^(m_p - A_i) never
// overflows and the largest weight never underflows.
template <int J>
__device__ __forceinline__ float weight_offset(const float *row, float zmin, uint32_t flags) {
    if (!(zmin < 1.f)) return 0.f;  // +inf: no fragment with alpha > 0
    const float full = absorbance_at<J>(row, clamp_depth(zmin), 0.f, flags & kLinear);
    return fmaxf(full - kStepCapLog2, 0.f);
}

// Stores one pixel's bin values (log2 units) into its padded shared row and,
// in the normalised resolve, folds in the weight offset: the row becomes
// A' = A - m_p with m_p from the pixel's nearest depth (every fragment then has
// A' >= 0 up to rounding, which the self-excluded clamp at 0 absorbs).
template <int J>
__device__ __forceinline__ void put_bins(float *row, float (&v)[1 << J], float zmin, uint32_t flags) {
    constexpr int C = 1 << J, V0 = Shape<J>::V0;
    auto put = [&]() {
        if constexpr (C % 4 == 0 && Shape<J>::LDV % 4 == 0 && V0 % 4 == 0) {  // 16-byte rows
#pragma unroll
            for (int q = 0; q < C / 4; ++q)
                reinterpret_cast<float4 *>(row + V0)[q] =
                    make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
#pragma unroll
            for (int i = 0; i < C; ++i) row[V0 + i] = v[i];
        }
        row[V0 - 1] = v[0];
        row[V0 + C] = v[C - 1];
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

// Step 2 accumulation, one pass over the fragments with bins scaled by a
// fixed 2^27 (SCALED = false) or by per-pixel scales s_p (SCALED = true, after
// count_pass).  Each fragment adds rint(s a f) and rint(s a (1-f)) to its bin
// with integer atomics and its depth to the pixel's nearest depth with a
// red.min.  Under the fixed scale the pass reports what the tile may need:
// bit 0, a bin word wrapped (seen from the atomics' return values); bit 1, a
// fragment's step is below 2^-7, where the fixed scale rounds it by more than
// 2^-21 of itself (phase_bins then looks at the pixels' totals).  Invalid
// fragments are counted in bad when COUNT.
template <int J, bool SCALED, bool COUNT>
__device__ __forceinline__ unsigned bins_pass(const Params &p, const Tile &T, unsigned *sF, unsigned *sG,
                                              unsigned *sZ, unsigned &bad) {
    constexpr int C = Shape<J>::C, LD = Shape<J>::LD, AMAX = Shape<J>::AMAX;
    constexpr float kFineStep = 1048576.f;  // 2^20: a step of 2^-7 under the fixed scale
    bool wrap = false, fine = false;
    for_each_group<kWithZ>(T.s, T.e, p, [&](auto &G) {
        constexpr int N = std::remove_reference_t<decltype(G)>::size;
        int lp[N];
        float sp[N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
            lp[k] = -1;
            if (G.v) {
                if (G.z[k] == G.z[k] && G.al[k] == G.al[k]) lp[k] = local_pixel(G.px[k], p, T);
                if (COUNT && lp[k] < 0) ++bad;
            }
        }
        // the group's scale reads, then its arithmetic, then its atomics
#pragma unroll
        for (int k = 0; k < N; ++k)
            sp[k] = SCALED ? (lp[k] >= 0 ? __uint_as_float(sF[lp[k] * LD + AMAX]) : 0.f) : kBinScale;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            if (lp[k] < 0) continue;
            const float a = step_of(clamp_alpha(G.al[k]));
            const float zc = clamp_depth(G.z[k]);
            const float s = zc * (float)C;  // exact: C is a power of two
            const Floor m = floor_small(s);
            const float f = s - m.f;
            const float as = a * sp[k];
            const unsigned vF = __float2uint_rn(as * f), vG = __float2uint_rn(as * (1.f - f));
            const unsigned oF = atomicAdd(&sF[lp[k] * LD + m.i], vF);
            const unsigned oG = atomicAdd(&sG[lp[k] * LD + m.i], vG);
            if (!SCALED) {
                wrap |= (oF + vF < oF) | (oG + vG < oG);
                fine |= as < kFineStep && a > 0.f;
            }
            if (a > 0.f) atomicMin(&sZ[lp[k]], __float_as_uint(zc));
        }
    });
    return (wrap ? 1u : 0u) | (fine ? 2u : 0u);
}

// Counting pass of the fallback: each pixel's fragment count c_p and largest
// clamped alpha (integer atomics on the padding words of its F row), then its
// scale s_p = 2^(30 - floor(log2(c_p a_max))), which keeps every bin sum below
// 2^32.  Ends with a barrier.
template <int J>
__device__ __forceinline__ void count_pass(const Params &p, const Tile &T, unsigned *sF) {
    constexpr int LD = Shape<J>::LD;
    constexpr int CNT = Shape<J>::CNT, AMAX = Shape<J>::AMAX, INV = Shape<J>::INV;
    for_each_group<0>(T.s, T.e, p, [&](auto &G) {
        constexpr int N = std::remove_reference_t<decltype(G)>::size;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int lp = G.v && G.al[k] == G.al[k] ? local_pixel(G.px[k], p, T) : -1;
            if (lp >= 0) {
                unsigned *row = sF + lp * LD;
                atomicAdd(&row[CNT], 1u);
                atomicMax(&row[AMAX], __float_as_uint(clamp_alpha(G.al[k])));
            }
        }
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
}

// Step 2 accumulation of one tile into its F and G bins (zeroed by the
// caller, nearest-depth words set to +inf).  The fixed-scale pass is tried
// first; if it reports a wrapped bin, or a step below 2^-7 in a pixel whose
// total step is below 2^-7 too, the bins are cleared and rebuilt with
// per-pixel scales.  (The fixed scale rounds every step by at most 2^-28
// absolute, so a pixel whose total is at least 2^-7 keeps its coefficients
// within 2^-21 of that total whatever its steps.)  Returns whether the
// per-pixel scales were used (the INV word of each pixel's F row then holds
// 1 / s_p).  Ends with a barrier.
template <int J>
__device__ __forceinline__ bool phase_bins(const Params &p, const Tile &T, unsigned *sF, unsigned *sG,
                                           unsigned *sZ, unsigned &bad) {
    const unsigned why = bins_pass<J, false, true>(p, T, sF, sG, sZ, bad);
    if (!__syncthreads_or(why)) return false;
    const int npx = p.g.tile_w * p.g.tile_h;
    if (!__syncthreads_or(why & 1u)) {  // only fine steps: do the pixels' totals resolve them?
        constexpr int C = Shape<J>::C, LD = Shape<J>::LD;
        bool small = false;
        for (int lp = threadIdx.x; lp < npx; lp += blockDim.x) {
            float tot = 0.f;  // sum of the bins in fixed-point units (a relative error of 2^-18 does not matter)
#pragma unroll 8
            for (int m = 0; m < C; ++m) tot += (float)sF[lp * LD + m] + (float)sG[lp * LD + m];
            small |= tot > 0.f && tot < 1048576.f;  // total step below 2^-7
        }
        if (!__syncthreads_or(small)) return false;
    }
    fill_zero(sF, (int)(2 * align16((size_t)npx * Shape<J>::LD * 4)));  // F and G planes are adjacent
    __syncthreads();
    count_pass<J>(p, T, sF);
    bins_pass<J, true, false>(p, T, sF, sG, sZ, bad);  // the nearest depths are already final
    __syncthreads();
    return true;
}

// Step 3 (§2.1).  Each pixel's row holds its bin values in log2 units minus
// the pixel's weight offset m_p, so v_i = 2^(m_p - A_i) = 2^-A'_i and
// w_i = alpha_i v_i; per pixel (R, G, B, W) += (c w, w) through the
// warp-segmented reduction into this warp's copy, and, when sS is given,
// S += a with a shared-memory atomic.  The own step removed under
// self-exclusion is -log2(1 - alpha), taken from the hardware log2 (its
// absolute error, ~2^-22, moves one fragment's exponent only), except when
// S needs the accurate step.
// CLAMP: exponents held to [0, 120] (the single pass, whose weight offset
// comes from another frame).
template <int J, bool COUNT, bool DEF = false, bool CLAMP = false>
__device__ __forceinline__ void phase_resolve(const Params &p, const Tile &T, const float *A2,
                                              float4 *accw, float *sS,
                                              unsigned &bad) {
    constexpr int LDV = Shape<J>::LDV;
    const uint32_t flags = DEF ? kDefaultFlags : p.flags;  // DEF: p.flags is the default
    const int npx = p.g.tile_w * p.g.tile_h;
    float4 *mine = accw + (threadIdx.x >> 5) * npx;
    for_each_group<kWithZ | kWithRGB>(T.s, T.e, p, [&](auto &G) {
        constexpr int N = std::remove_reference_t<decltype(G)>::size;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            const int lp = G.v && G.z[k] == G.z[k] && G.al[k] == G.al[k] ? local_pixel(G.px[k], p, T) : -1;
            if (COUNT && G.v && lp < 0) ++bad;
            // a lane without a valid fragment evaluates pixel 0 and adds nothing
            const int l = lp >= 0 ? lp : 0;
            const float ac = clamp_alpha(G.al[k]);  // 0 for NaN
            float a = 0.f, a2;
            if (sS) {
                a = step_of(ac);
                a2 = a * kLog2e;
            } else {
                a2 = -lg2(1.f - ac);
            }
            float Ah = absorbance_at<J>(A2 + l * LDV, clamp_depth(G.z[k]), a2, flags);
            if constexpr (CLAMP) Ah = fminf(fmaxf(Ah, 0.f), 120.f);
            const float w = ac * ex2(-Ah);
            if (sS && lp >= 0) atomicAdd(&sS[l], a);
            warp_accumulate(mine, lp, make_float4(G.r[k] * w, G.g[k] * w, G.b[k] * w, w));
        }
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
    const float T = ex2(-S * kLog2e);
    // 1 - T; for small S the series S (1 - S/2) (error below S^3/6 < 3e-10)
    const float cover = S < 0.0009765625f ? S * fmaf(-0.5f, S, 1.f) : 1.f - T;
    float4 o;
    if (p.flags & kNormalized) {
        if (W > 0.f) {
            const float k = W >= 1.17549435e-38f ? cover * rcp(W) : cover / W;  // (subnormal W)
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

// Every region starts on a 16-byte boundary (float4 row reads and writes).
template <int J> struct Layout {
    static constexpr size_t plane(int npx) { return align16((size_t)npx * Shape<J>::LD * 4); }
    static constexpr size_t vplane(int npx) { return align16((size_t)npx * Shape<J>::LDV * 4); }
    static constexpr size_t words(int npx) { return align16((size_t)npx * 4); }
    // the warps' accumulators; the same region stages a tile's coefficient
    // rows on their way to or from global memory, so it holds the larger of
    // the two (an FP32 row is wider than the accumulators from J = 6 on)
    static constexpr size_t accw(int npx) {
        return (size_t)npx * (kWarps * 16 > Shape<J>::C * 4 ? kWarps * 16 : Shape<J>::C * 4);
    }
    // build: F and G bins + nearest-depth words
    static constexpr size_t build(int npx) { return 2 * plane(npx) + words(npx); }
    // fused: F and G bins, replaced after the build by the bin values, the
    // warps' accumulators and the S words; then the nearest-depth words
    static constexpr size_t region(int npx) {
        return 2 * plane(npx) > vplane(npx) + accw(npx) + words(npx)
                   ? 2 * plane(npx)
                   : vplane(npx) + accw(npx) + words(npx);
    }
    static constexpr size_t fused(int npx) { return region(npx) + words(npx); }
    // resolve: bin values + warps' accumulators + S words
    static constexpr size_t resolve(int npx) { return vplane(npx) + accw(npx) + words(npx); }
};

}  // namespace wt
