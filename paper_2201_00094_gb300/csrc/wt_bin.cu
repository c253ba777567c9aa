// Steps before the coefficient build: grouping an unordered fragment stream
// by screen tile, and the per-pixel depth bounds of §2.1 step 1 with the
// normalisation of depth into them.
//
// Binning is a stable least-significant-digit radix sort of the fragments by
// tile id (row-major tiles of the descriptor), 8 bits per pass: two passes for
// up to 65536 tiles.  A pass is three kernels:
//   * a histogram of the pass's digit over each block's 8192 consecutive
//     fragments (shared-memory counters), stored digit-major [257][blocks];
//   * an exclusive scan of that matrix along each digit row, and of the row
//     totals over the digits: fragment (digit d, block b) then starts at
//     base[d] + M[d][b] in the pass's output;
//   * a scatter: each block ranks its fragments by digit (match.any within a
//     warp, per-warp counters in shared memory, in input order, so the sort is
//     stable), places each field in shared memory in digit order and writes
//     it out: a block's fragments of one digit are a contiguous run of the
//     output, so the stores are coalesced however random the input order is.
// The scatter of a pass that is not the last also writes the next pass's
// digit as one byte per fragment, so that the next histogram reads one byte.
// Fragments whose pixel id is outside the image fall into a 257th bucket that
// is never written, and are counted.  Because every pass is stable, the
// fragments of a tile come out in their input order: the result is
// deterministic.  tile_offsets is read off the sorted stream (a tile starts
// where the tile id changes).
//
// Depth bounds run per tile over a tile-grouped stream: shared-memory min/max
// per pixel, one store per pixel.  Depth is compared through an order-
// preserving map of the float bits to unsigned integers, so negative depths
// order correctly.
#include "wt.h"
#include "wt_internal.h"
#include "wt_trace.h"
#include "wt_tile.cuh"

namespace wt {

unsigned long long *error_word();  // wt_api.cu

namespace {

// floor(x / d) for every 32-bit x by a multiply-high (Granlund & Montgomery
// 1994, round-up method): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// t = mulhi(x, m), q = (t + ((x - t) >> min(l, 1))) >> max(l - 1, 0).
struct FastDiv {
    uint32_t m;
    int s1, s2;
};
FastDiv make_fastdiv(uint32_t d) {
    int l = 0;
    while ((1ull << l) < d) ++l;
    FastDiv f;
    f.m = (uint32_t)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t x, const FastDiv &f) {
    const uint32_t t = __umulhi(x, f.m);
    return (t + ((x - t) >> f.s1)) >> f.s2;
}

struct BinGeom {
    uint32_t width, tile_w, tile_h, ntx;
    int64_t P;
    FastDiv dw, dtw, dth;
};

// Row-major tile index of a pixel id inside the image.
__device__ __forceinline__ uint32_t tile_of_pixel(uint32_t px, const BinGeom &g) {
    const uint32_t y = fdiv(px, g.dw), x = px - y * g.width;
    return fdiv(y, g.dth) * g.ntx + fdiv(x, g.dtw);
}

constexpr int kRT = 512;             // threads of a sorting block
constexpr int kRW = kRT / 32;        // its warps
constexpr int kRI = 16;              // fragments per thread
constexpr int kRTile = kRT * kRI;    // fragments per block
constexpr int kRD = 257;             // 256 digits + the bucket of dropped fragments

// Shared memory of a scatter block (bytes, dynamic): the run starts of the
// digits in the output, the per-warp digit counts, the digits' block-local
// starts, the staged field, the output index of each block-local position and
// (first of several passes) the next pass's digit.
struct ScatterSmem {
    static constexpr size_t gdst = 0;
    static constexpr size_t wcnt = gdst + 256 * 8;
    static constexpr size_t lstart = wcnt + (size_t)kRW * kRD * 4;
    static constexpr size_t stage = (lstart + kRD * 4 + 15) & ~size_t(15);
    static constexpr size_t sdst = stage + (size_t)kRTile * 4;
    static constexpr size_t snext = sdst + (size_t)kRTile * 4;
    static constexpr size_t bytes(bool next) { return snext + (next ? (size_t)kRTile : 16); }
};

struct BinIn {
    const uint32_t *pixel;
    const float *z, *alpha, *r, *g, *b;
};
struct BinOut {
    uint32_t *pixel;
    float *z, *alpha, *r, *g, *b;
};

// Digit of pass `pass` of a fragment: (tile >> 8 pass) & 255 for a pixel in
// the image, 256 otherwise.
__device__ __forceinline__ int first_digit(uint32_t px, const BinGeom &g, int pass) {
    if ((int64_t)px >= g.P) return 256;
    return (int)((tile_of_pixel(px, g) >> (8 * pass)) & 255u);
}

// Histogram of the pass's digit over each block's fragments, stored
// digit-major: M[d * nb + block].  FIRST: the digit comes from the pixel id
// (dropped fragments counted into err); otherwise from the byte array written
// by the previous pass, over the kept fragments.  Each thread reads its 16
// keys as whole 16-byte vectors where the block's range allows.
template <bool FIRST>
__global__ void __launch_bounds__(kRT) k_bin_hist(BinGeom g, int64_t n, const unsigned long long *kept,
                                                  int pass, int nb, const uint32_t *__restrict__ pixel,
                                                  const uint8_t *__restrict__ dig, unsigned *__restrict__ M,
                                                  unsigned long long *err) {
    __shared__ unsigned h[kRD];
    for (int d = threadIdx.x; d < kRD; d += kRT) h[d] = 0u;
    __syncthreads();
    const int64_t ne = FIRST ? n : (int64_t)*kept;
    const int64_t i0 = (int64_t)blockIdx.x * kRTile + (int64_t)threadIdx.x * kRI;  // this thread's 16 keys
    unsigned bad = 0;
    if constexpr (FIRST) {
        uint32_t key[kRI];
        if (i0 + kRI <= ne) {  // i0 is a multiple of 16 elements: 16-byte aligned
#pragma unroll
            for (int j = 0; j < kRI; j += 4) {
                const uint4 u = *reinterpret_cast<const uint4 *>(pixel + i0 + j);
                key[j] = u.x, key[j + 1] = u.y, key[j + 2] = u.z, key[j + 3] = u.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kRI; ++j) key[j] = i0 + j < ne ? pixel[i0 + j] : 0u;
        }
#pragma unroll
        for (int j = 0; j < kRI; ++j) {
            if (i0 + j >= ne) break;
            const int d = first_digit(key[j], g, pass);
            if (d == 256) ++bad;
            atomicAdd(&h[d], 1u);
        }
        flush_bad(bad, err);
    } else {
        uint4 u = make_uint4(0u, 0u, 0u, 0u);
        if (i0 + kRI <= ne) {
            u = *reinterpret_cast<const uint4 *>(dig + i0);
        } else {
            uint8_t *ub = reinterpret_cast<uint8_t *>(&u);
            for (int j = 0; j < kRI; ++j) ub[j] = i0 + j < ne ? dig[i0 + j] : 0;
        }
        const uint32_t word[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int j = 0; j < kRI; ++j) {
            if (i0 + j >= ne) break;
            atomicAdd(&h[(word[j >> 2] >> (8 * (j & 3))) & 255u], 1u);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRD; d += kRT) M[(int64_t)d * nb + blockIdx.x] = h[d];
}

// Exclusive scan of one digit row of M in place (one block per digit), in
// rounds of 1024 consecutive entries; the row's total goes to rowsum[d].
__global__ void __launch_bounds__(1024) k_bin_rows(unsigned *__restrict__ M, int nb,
                                                   unsigned long long *__restrict__ rowsum) {
    __shared__ unsigned warp_sum[32];
    unsigned *row = M + (int64_t)blockIdx.x * nb;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const unsigned v = i < nb ? row[i] : 0u;
        unsigned x = v;  // inclusive scan within the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sum[w] = x;
        __syncthreads();
        if (w == 0) {
            unsigned s = warp_sum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_sum[lane] = s;  // inclusive over warps
        }
        __syncthreads();
        const unsigned before = (w ? warp_sum[w - 1] : 0u) + x - v;
        if (i < nb) row[i] = (unsigned)(carry + before);
        carry += warp_sum[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) rowsum[blockIdx.x] = carry;
}

// Exclusive scan of the 256 row totals into base[d]; kept = their sum (the
// fragments that pass through the sort).
__global__ void __launch_bounds__(256) k_bin_bases(const unsigned long long *__restrict__ rowsum,
                                                   unsigned long long *__restrict__ base,
                                                   unsigned long long *__restrict__ kept) {
    __shared__ unsigned long long s[256];
    const int t = threadIdx.x;
    s[t] = rowsum[t];
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        const unsigned long long y = t >= o ? s[t - o] : 0ull;
        __syncthreads();
        s[t] += y;
        __syncthreads();
    }
    base[t] = s[t] - rowsum[t];
    if (t == 255) *kept = s[255];
}

// One pass of the sort: ranks the block's fragments by digit (stable), then
// moves every field through shared memory into digit order and out to its
// run.  FIRST: digits from the pixel ids; LAST: no next digit to write.  The
// keys of all the thread's fragments are loaded before the ranking, and the
// next field's values are loaded while the current one is written out.
template <bool FIRST, bool LAST, bool RGB>
__global__ void __launch_bounds__(kRT, 2) k_bin_scatter(BinGeom g, int64_t n, const unsigned long long *kept,
                                                        int pass, int nb, BinIn in, const uint8_t *__restrict__ dig_in,
                                                        BinOut out, uint8_t *__restrict__ dig_out,
                                                        const unsigned *__restrict__ M,
                                                        const unsigned long long *__restrict__ base) {
    extern __shared__ __align__(16) unsigned char smem[];
    using L = ScatterSmem;
    // where this block's run of each digit starts in the output
    unsigned long long *gdst = reinterpret_cast<unsigned long long *>(smem + L::gdst);
    // per-warp digit counts, then exclusive offsets over warps: wcnt[w][d] at w * kRD + d
    unsigned(*wcnt)[kRD] = reinterpret_cast<unsigned(*)[kRD]>(smem + L::wcnt);
    unsigned *lstart = reinterpret_cast<unsigned *>(smem + L::lstart);  // block-local start of each digit's run
    uint32_t *stage = reinterpret_cast<uint32_t *>(smem + L::stage);
    uint32_t *sdst = reinterpret_cast<uint32_t *>(smem + L::sdst);  // output index of each block-local position
    uint8_t *snext = smem + L::snext;  // the next pass's digit (first of several passes)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRW * kRD; i += kRT) (&wcnt[0][0])[i] = 0u;
    const int64_t ne = FIRST ? n : (int64_t)*kept;
    const int64_t b0 = (int64_t)blockIdx.x * kRTile + w * (32 * kRI) + lane;  // fragment k at b0 + 32 k
    // the keys (FIRST: the pixel ids, which are also the first field moved)
    uint32_t val[kRI];
#pragma unroll
    for (int k = 0; k < kRI; ++k) {
        const int64_t i = b0 + 32 * k;
        val[k] = i < ne ? (FIRST ? in.pixel[i] : (uint32_t)dig_in[i]) : 0xffffffffu;
    }
    __syncthreads();
    unsigned lt;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(lt));
    unsigned pos[kRI];
    // rank within the warp's fragments of the same digit, in input order, kept
    // as rank | digit << 12 | next << 21 (the first pass keeps the next pass's
    // digit, from the same tile id)
#pragma unroll
    for (int k = 0; k < kRI; ++k) {
        int d = 256;
        uint32_t nx = 0;
        if (b0 + 32 * k < ne) {
            if constexpr (FIRST) {
                if ((int64_t)val[k] < g.P) {
                    const uint32_t t = tile_of_pixel(val[k], g);
                    d = (int)((t >> (8 * pass)) & 255u);
                    nx = (t >> (8 * pass + 8)) & 255u;
                }
            } else {
                d = (int)val[k];
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int leader = __ffs(peers) - 1;
        unsigned old = 0;
        if (lane == leader) {
            old = wcnt[w][d];
            wcnt[w][d] = old + __popc(peers);
        }
        old = __shfl_sync(0xffffffffu, old, leader);
        pos[k] = (old + __popc(peers & lt)) | ((unsigned)d << 12) | (nx << 21);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRD; d += kRT) {
        unsigned run = 0;
        for (int ww = 0; ww < kRW; ++ww) {
            const unsigned c = wcnt[ww][d];
            wcnt[ww][d] = run;
            run += c;
        }
        lstart[d] = run;  // the digit's block total, scanned below
    }
    __syncthreads();
    if (w == 0) {  // exclusive scan of the 257 totals: lane l owns digits 9 l .. 9 l + 8
        unsigned v[9], sum = 0;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const int d = 9 * lane + j;
            v[j] = d < kRD ? lstart[d] : 0u;
            sum += v[j];
        }
        unsigned x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        unsigned run = x - sum;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const int d = 9 * lane + j;
            if (d < kRD) lstart[d] = run;
            run += v[j];
        }
    }
    for (int d = threadIdx.x; d < 256; d += kRT) gdst[d] = base[d] + M[(int64_t)d * nb + blockIdx.x];
    __syncthreads();
    // block-local positions (a position below nvalid is a kept fragment) and
    // the output index of each
#pragma unroll
    for (int k = 0; k < kRI; ++k) {
        const int d = (int)((pos[k] >> 12) & 511u);
        const unsigned nx = pos[k] >> 21;
        const unsigned within = (pos[k] & 4095u) + wcnt[w][d];  // rank in the block's run of digit d
        pos[k] = within + lstart[d];
        if (d < 256) {
            sdst[pos[k]] = (uint32_t)(gdst[d] + within);
            if constexpr (FIRST && !LAST) snext[pos[k]] = (uint8_t)nx;
        }
    }
    const unsigned nvalid = lstart[256];  // the block's fragments that are written
    if (!FIRST) {  // the first field, the pixel ids
#pragma unroll
        for (int k = 0; k < kRI; ++k)
            if (pos[k] < nvalid) val[k] = in.pixel[b0 + 32 * k];
    }
    __syncthreads();
    const uint32_t *src[6] = {in.pixel, reinterpret_cast<const uint32_t *>(in.z),
                              reinterpret_cast<const uint32_t *>(in.alpha), reinterpret_cast<const uint32_t *>(in.r),
                              reinterpret_cast<const uint32_t *>(in.g), reinterpret_cast<const uint32_t *>(in.b)};
    uint32_t *dst[6] = {out.pixel, reinterpret_cast<uint32_t *>(out.z), reinterpret_cast<uint32_t *>(out.alpha),
                        reinterpret_cast<uint32_t *>(out.r), reinterpret_cast<uint32_t *>(out.g),
                        reinterpret_cast<uint32_t *>(out.b)};
    constexpr int kFields = RGB ? 6 : 3;
#pragma unroll
    for (int f = 0; f < kFields; ++f) {
#pragma unroll
        for (int k = 0; k < kRI; ++k)
            if (pos[k] < nvalid) stage[pos[k]] = val[k];
        __syncthreads();
        if (f + 1 < kFields) {  // the next field's loads, in flight during the write-out
#pragma unroll
            for (int k = 0; k < kRI; ++k)
                if (pos[k] < nvalid) val[k] = src[f + 1][b0 + 32 * k];
        }
        for (unsigned q = threadIdx.x; q < nvalid; q += kRT) {
            const uint32_t o = sdst[q];
            const uint32_t v = stage[q];
            dst[f][o] = v;
            if (!LAST && f == 0)
                dig_out[o] = FIRST ? snext[q] : (uint8_t)((tile_of_pixel(v, g) >> (8 * pass + 8)) & 255u);
        }
        __syncthreads();
    }
}

// tile_offsets from the sorted stream: position i opens the tiles after the
// previous fragment's tile up to its own; position kept closes the rest.
// Each thread takes 8 consecutive positions (two 16-byte loads); the tile
// before its first one comes from the lane below (lane 0 reads it).
constexpr int kOffPer = 8;
__global__ void __launch_bounds__(256) k_bin_offsets(BinGeom g, int64_t ntiles, const uint32_t *__restrict__ pixel,
                                                     const unsigned long long *kept, int64_t *__restrict__ off) {
    const int64_t K = (int64_t)*kept;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * kOffPer;
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31)) * kOffPer; b <= K; b += stride) {
        const int64_t i0 = b + (int64_t)lane * kOffPer;
        int64_t t[kOffPer];
        if (i0 + kOffPer <= K) {  // i0 is a multiple of 8 elements: 16-byte aligned
            const uint4 u0 = *reinterpret_cast<const uint4 *>(pixel + i0);
            const uint4 u1 = *reinterpret_cast<const uint4 *>(pixel + i0 + 4);
            const uint32_t px[kOffPer] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
            for (int j = 0; j < kOffPer; ++j) t[j] = (int64_t)tile_of_pixel(px[j], g);
        } else {
#pragma unroll
            for (int j = 0; j < kOffPer; ++j)
                t[j] = i0 + j < K ? (int64_t)tile_of_pixel(pixel[i0 + j], g) : ntiles;
        }
        int64_t tp = __shfl_up_sync(0xffffffffu, t[kOffPer - 1], 1);
        if (lane == 0) tp = i0 > 0 ? (int64_t)tile_of_pixel(pixel[i0 - 1], g) : -1;
#pragma unroll
        for (int j = 0; j < kOffPer; ++j) {
            const int64_t i = i0 + j;
            if (i <= K)
                for (int64_t u = tp + 1; u <= t[j]; ++u) off[u] = i;
            tp = t[j];
        }
    }
}

// order-preserving map of float bits to unsigned (and back)
__device__ __forceinline__ unsigned order_key(float x) {
    const unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_key(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Per-pixel min and max depth of a tile's valid fragments (z and alpha not
// NaN, pixel inside the tile); +inf / -inf for pixels with none.
__global__ void __launch_bounds__(kThreads) k_depth_bounds(Params p, float *__restrict__ zlo,
                                                           float *__restrict__ zhi) {
    __shared__ unsigned slo[kMaxTilePx], shi[kMaxTilePx];
    const int npx = p.g.tile_w * p.g.tile_h;
    for (int i = threadIdx.x; i < npx; i += blockDim.x) {
        slo[i] = order_key(__int_as_float(0x7f800000));
        shi[i] = order_key(__int_as_float(0xff800000));
    }
    const Tile T = tile_of(p, blockIdx.x, true);
    __syncthreads();
    unsigned bad = 0;
    for_each_group<kWithZ>(T.s, T.e, p, [&](auto &G) {
        constexpr int N = std::remove_reference_t<decltype(G)>::size;
#pragma unroll
        for (int k = 0; k < N; ++k) {
            if (!G.v) continue;
            const int lp = G.z[k] == G.z[k] && G.al[k] == G.al[k] ? local_pixel(G.px[k], p, T) : -1;
            if (lp < 0) {
                ++bad;
                continue;
            }
            const unsigned key = order_key(G.z[k]);
            atomicMin(&slo[lp], key);
            atomicMax(&shi[lp], key);
        }
    });
    flush_bad(bad, p.err);
    __syncthreads();
    const int lp = threadIdx.x;
    if (lp >= npx) return;
    const int64_t gp = global_pixel(p, T, lp);
    if (gp < 0) return;
    zlo[gp] = from_key(slo[lp]);
    zhi[gp] = from_key(shi[lp]);
}

// z_out = (z - zlo_p) / (zhi_p - zlo_p) for the fragment's pixel p, 0 when the
// range is empty or not finite; fragments with a bad pixel id or NaN keep NaN.
__device__ __forceinline__ float normalized_depth(uint32_t px, float zi, int64_t P, const float *__restrict__ zlo,
                                                  const float *__restrict__ zhi) {
    float o = __int_as_float(0x7fc00000);
    if ((int64_t)px < P && zi == zi) {
        const float lo = zlo[px], range = zhi[px] - lo;
        o = range > 0.f && range < __int_as_float(0x7f800000) ? (zi - lo) / range : 0.f;
    }
    return o;
}
__global__ void __launch_bounds__(256) k_normalize_depth(int64_t n, int64_t P, const uint32_t *__restrict__ pixel,
                                                         const float *z, const float *__restrict__ zlo,
                                                         const float *__restrict__ zhi, float *z_out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        z_out[i] = normalized_depth(pixel[i], z[i], P, zlo, zhi);
}
// The same four fragments per thread, for 16-byte aligned pixel, z and z_out:
// one vector load per array and four independent bound reads in flight; the
// thread past the last whole group takes the last n mod 4 fragments.
__global__ void __launch_bounds__(256) k_normalize_depth4(int64_t n, int64_t P, const uint32_t *__restrict__ pixel,
                                                          const float *z, const float *__restrict__ zlo,
                                                          const float *__restrict__ zhi, float *z_out) {
    const int64_t n4 = n >> 2;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q <= n4;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (q < n4) {
            const uint4 pv = reinterpret_cast<const uint4 *>(pixel)[q];
            const float4 zv = reinterpret_cast<const float4 *>(z)[q];
            float4 o;
            o.x = normalized_depth(pv.x, zv.x, P, zlo, zhi);
            o.y = normalized_depth(pv.y, zv.y, P, zlo, zhi);
            o.z = normalized_depth(pv.z, zv.z, P, zlo, zhi);
            o.w = normalized_depth(pv.w, zv.w, P, zlo, zhi);
            reinterpret_cast<float4 *>(z_out)[q] = o;
        } else {
            for (int64_t i = 4 * n4; i < n; ++i) z_out[i] = normalized_depth(pixel[i], z[i], P, zlo, zhi);
        }
    }
}

int grid_for(int64_t n) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (n + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

bool aligned_to(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

wt_status check_geom(const wt_desc *d) {
    if (!d || d->width < 1 || d->height < 1 || d->tile_w < 1 || d->tile_h < 1) return WT_ERR_ARG;
    if ((int64_t)d->width * d->height >= (int64_t(1) << 31)) return WT_ERR_ARG;
    if ((int64_t)d->tile_w * d->tile_h > kMaxTilePx) return WT_ERR_ARG;
    return WT_OK;
}

BinGeom bin_geom(const wt_desc *d) {
    BinGeom g;
    g.width = (uint32_t)d->width;
    g.tile_w = (uint32_t)d->tile_w;
    g.tile_h = (uint32_t)d->tile_h;
    g.ntx = (uint32_t)((d->width + d->tile_w - 1) / d->tile_w);
    g.P = (int64_t)d->width * d->height;
    g.dw = make_fastdiv(g.width);
    g.dtw = make_fastdiv(g.tile_w);
    g.dth = make_fastdiv(g.tile_h);
    return g;
}

int64_t tiles_of(const wt_desc *d) {
    return (int64_t)((d->width + d->tile_w - 1) / d->tile_w) * ((d->height + d->tile_h - 1) / d->tile_h);
}

// Radix passes of 8 bits that the tile ids need (1 to 4).
int sort_passes(int64_t ntiles) {
    int bits = 1;
    while (bits < 32 && (int64_t(1) << bits) < ntiles) ++bits;
    return (bits + 7) / 8;
}

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// Workspace layout (256-byte aligned regions): the digit matrix [257][nb]
// (unsigned), the row totals and digit bases (256 each), the kept count, then
// for two passes or more one intermediate structure-of-arrays stream (six
// arrays of n) and one byte per fragment for the next digit, and for three or
// more a second of each (the passes alternate between them).
struct BinWorkspace {
    unsigned *M;
    unsigned long long *rowsum, *base, *kept;
    char *soa[2];
    uint8_t *dig[2];
};
size_t workspace_layout(int64_t ntiles, int64_t n, char *ws, BinWorkspace *out) {
    const int64_t nb = (n + kRTile - 1) / kRTile;
    const int passes = sort_passes(ntiles);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += up256(bytes);
        return ws ? ws + at : nullptr;
    };
    char *M = take((size_t)kRD * (size_t)(nb > 0 ? nb : 1) * 4);
    char *rowsum = take(256 * 8), *base = take(256 * 8), *kept = take(8);
    char *soa[2] = {nullptr, nullptr};
    char *dig[2] = {nullptr, nullptr};
    for (int k = 0; k < 2; ++k) {
        if (passes >= 2 + k) {
            soa[k] = take((size_t)n * 24);
            dig[k] = take((size_t)n);
        }
    }
    if (out) {
        out->M = reinterpret_cast<unsigned *>(M);
        out->rowsum = reinterpret_cast<unsigned long long *>(rowsum);
        out->base = reinterpret_cast<unsigned long long *>(base);
        out->kept = reinterpret_cast<unsigned long long *>(kept);
        for (int k = 0; k < 2; ++k) {
            out->soa[k] = soa[k];
            out->dig[k] = reinterpret_cast<uint8_t *>(dig[k]);
        }
    }
    return o;
}

// The six arrays of an intermediate stream in a workspace region.
BinOut soa_arrays(char *base, int64_t n) {
    BinOut o;
    o.pixel = reinterpret_cast<uint32_t *>(base);
    o.z = reinterpret_cast<float *>(base + (size_t)n * 4);
    o.alpha = reinterpret_cast<float *>(base + (size_t)n * 8);
    o.r = reinterpret_cast<float *>(base + (size_t)n * 12);
    o.g = reinterpret_cast<float *>(base + (size_t)n * 16);
    o.b = reinterpret_cast<float *>(base + (size_t)n * 20);
    return o;
}

template <bool FIRST, bool LAST>
void launch_scatter(bool rgb, int nb, cudaStream_t s, const BinGeom &g, int64_t n, const unsigned long long *kept,
                    int pass, const BinIn &in, const uint8_t *dig_in, const BinOut &out, uint8_t *dig_out,
                    const unsigned *M, const unsigned long long *base) {
    const size_t bytes = ScatterSmem::bytes(FIRST && !LAST);
    if (rgb) {
        cudaFuncSetAttribute(k_bin_scatter<FIRST, LAST, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        k_bin_scatter<FIRST, LAST, true><<<nb, kRT, bytes, s>>>(g, n, kept, pass, nb, in, dig_in, out, dig_out, M,
                                                                base);
    } else {
        cudaFuncSetAttribute(k_bin_scatter<FIRST, LAST, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bytes);
        k_bin_scatter<FIRST, LAST, false><<<nb, kRT, bytes, s>>>(g, n, kept, pass, nb, in, dig_in, out, dig_out, M,
                                                                 base);
    }
}

}  // namespace
}  // namespace wt

using namespace wt;

extern "C" size_t wt_bin_workspace_bytes(const wt_desc *desc, int64_t n) {
    if (check_geom(desc) != WT_OK || n < 0) return 0;
    return workspace_layout(tiles_of(desc), n, nullptr, nullptr);
}

extern "C" wt_status wt_bin(const wt_desc *desc, const wt_frags *in, uint32_t *pixel_out, float *z_out,
                            float *alpha_out, float *r_out, float *g_out, float *b_out,
                            int64_t *tile_offsets_out, void *workspace, size_t workspace_bytes,
                            wt_stream stream) {
    WT_TRACE();
    wt_status st = check_geom(desc);
    if (st != WT_OK) return st;
    if (!in || in->n < 0 || !tile_offsets_out || !workspace) return WT_ERR_ARG;
    if (!aligned_to(workspace, 256) || !aligned_to(tile_offsets_out, 8)) return WT_ERR_ARG;
    if (workspace_bytes < wt_bin_workspace_bytes(desc, in->n)) return WT_ERR_ARG;
    const bool rgb = in->r != nullptr;
    if (rgb != (in->g != nullptr) || rgb != (in->b != nullptr)) return WT_ERR_ARG;
    if (in->n > 0) {
        const void *need[6] = {in->pixel, in->z, in->alpha, pixel_out, z_out, alpha_out};
        for (const void *p : need)
            if (!p) return WT_ERR_ARG;
        if (rgb && (!r_out || !g_out || !b_out)) return WT_ERR_ARG;
        if (!aligned_to(in->pixel, 16) || !aligned_to(pixel_out, 16)) return WT_ERR_ARG;  // vector loads
    }
    unsigned long long *err = error_word();
    if (!err) return WT_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t nt = tiles_of(desc), n = in->n;
    BinWorkspace W;
    workspace_layout(nt, n, static_cast<char *>(workspace), &W);
    const BinGeom g = bin_geom(desc);
    const int passes = sort_passes(nt);
    if (n >= (int64_t(1) << 32)) return WT_ERR_ARG;  // output indices are 32-bit
    const int64_t nb64 = (n + kRTile - 1) / kRTile;
    const int nb = (int)nb64;
    if (nb > 0) {
        const BinIn src{in->pixel, in->z, in->alpha, in->r, in->g, in->b};
        const BinOut dst{pixel_out, z_out, alpha_out, r_out, g_out, b_out};
        BinIn cur = src;
        const uint8_t *dig_in = nullptr;
        for (int pass = 0; pass < passes; ++pass) {
            const bool first = pass == 0, last = pass == passes - 1;
            if (first)
                k_bin_hist<true><<<nb, kRT, 0, s>>>(g, n, W.kept, pass, nb, in->pixel, nullptr, W.M, err);
            else
                k_bin_hist<false><<<nb, kRT, 0, s>>>(g, n, W.kept, pass, nb, nullptr, dig_in, W.M, err);
            k_bin_rows<<<256, 1024, 0, s>>>(W.M, nb, W.rowsum);
            k_bin_bases<<<1, 256, 0, s>>>(W.rowsum, W.base, W.kept);
            const BinOut to = last ? dst : soa_arrays(W.soa[pass & 1], n);
            uint8_t *dig_out = last ? nullptr : W.dig[pass & 1];
            if (first && last) launch_scatter<true, true>(rgb, nb, s, g, n, W.kept, pass, cur, dig_in, to, dig_out, W.M, W.base);
            else if (first) launch_scatter<true, false>(rgb, nb, s, g, n, W.kept, pass, cur, dig_in, to, dig_out, W.M, W.base);
            else if (last) launch_scatter<false, true>(rgb, nb, s, g, n, W.kept, pass, cur, dig_in, to, dig_out, W.M, W.base);
            else launch_scatter<false, false>(rgb, nb, s, g, n, W.kept, pass, cur, dig_in, to, dig_out, W.M, W.base);
            cur = BinIn{to.pixel, to.z, to.alpha, to.r, to.g, to.b};
            dig_in = dig_out;
        }
    } else if (cudaMemsetAsync(W.kept, 0, 8, s) != cudaSuccess) {
        return WT_ERR_CUDA;
    }
    k_bin_offsets<<<grid_for((n + kOffPer) / kOffPer), 256, 0, s>>>(g, nt, pixel_out, W.kept, tile_offsets_out);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

extern "C" wt_status wt_depth_bounds(const wt_desc *desc, const wt_frags *frags, float *zlo, float *zhi,
                                     wt_stream stream) {
    WT_TRACE();
    wt_status st = check_geom(desc);
    if (st != WT_OK) return st;
    if (!frags || frags->n < 0 || !frags->tile_offsets || !zlo || !zhi) return WT_ERR_ARG;
    if (!aligned_to(frags->tile_offsets, 8)) return WT_ERR_ARG;
    const void *req[3] = {frags->pixel, frags->z, frags->alpha};
    for (const void *p : req)
        if ((frags->n > 0 && !p) || !aligned_to(p, 16)) return WT_ERR_ARG;
    unsigned long long *err = error_word();
    if (!err) return WT_ERR_CUDA;
    Params p{};
    p.g.width = desc->width;
    p.g.height = desc->height;
    p.g.tile_w = desc->tile_w;
    p.g.tile_h = desc->tile_h;
    p.g.ntx = (desc->width + desc->tile_w - 1) / desc->tile_w;
    set_row_division(p);
    p.n = frags->n;
    p.pixel = frags->pixel;
    p.z = frags->z;
    p.alpha = frags->alpha;
    p.off = frags->tile_offsets;
    p.err = err;
    const int64_t nt = tiles_of(desc);
    k_depth_bounds<<<(unsigned)nt, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(p, zlo, zhi);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

extern "C" wt_status wt_normalize_depth(const wt_desc *desc, const wt_frags *frags, const float *zlo,
                                        const float *zhi, float *z_out, wt_stream stream) {
    WT_TRACE();
    wt_status st = check_geom(desc);
    if (st != WT_OK) return st;
    if (!frags || frags->n < 0 || !zlo || !zhi) return WT_ERR_ARG;
    if (frags->n > 0 && (!frags->pixel || !frags->z || !z_out)) return WT_ERR_ARG;
    if (frags->n == 0) return WT_OK;
    const int64_t P = (int64_t)desc->width * desc->height;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (aligned_to(frags->pixel, 16) && aligned_to(frags->z, 16) && aligned_to(z_out, 16))
        k_normalize_depth4<<<grid_for(frags->n / 4 + 1), 256, 0, s>>>(frags->n, P, frags->pixel, frags->z, zlo, zhi,
                                                                        z_out);
    else
        k_normalize_depth<<<grid_for(frags->n), 256, 0, s>>>(frags->n, P, frags->pixel, frags->z, zlo, zhi, z_out);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}
