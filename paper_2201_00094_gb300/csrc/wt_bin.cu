// Steps before the coefficient build: grouping an unordered fragment stream
// by screen tile, and the per-pixel depth bounds of §2.1 step 1 with the
// normalisation of depth into them.
//
// Binning is a counting sort by tile id (row-major tiles of the descriptor):
// a histogram pass, one exclusive scan of the tile counts into tile_offsets, a
// scatter pass in which every fragment takes the next slot of its tile and is
// staged there as one record, and a pass that unpacks the records in order
// into the output arrays.  When the tile counters fit in shared memory, each
// block counts and ranks its own chunk of the stream with shared atomics;
// otherwise the counts and slots come from global atomics.  Fragments whose pixel id is outside the image are dropped and
// counted.  The order of the
// fragments inside a tile is that of the atomics: the build does not depend on
// it (its sums are integer), the resolve's FP32 sums may differ in the last
// bits between runs.
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

struct BinGeom {
    int width, height, tile_w, tile_h, ntx;
    int64_t P;
};

// Row-major tile index of a pixel id, or -1 outside the image.
__device__ __forceinline__ int64_t tile_index(uint32_t px, const BinGeom &g) {
    if ((int64_t)px >= g.P) return -1;
    const uint32_t y = px / (uint32_t)g.width, x = px - y * (uint32_t)g.width;
    return (int64_t)(y / (uint32_t)g.tile_h) * g.ntx + x / (uint32_t)g.tile_w;
}

__global__ void __launch_bounds__(256) k_bin_count(BinGeom g, int64_t n, const uint32_t *__restrict__ pixel,
                                                   unsigned *__restrict__ counts, unsigned long long *err) {
    unsigned bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = tile_index(pixel[i], g);
        if (t < 0) ++bad;
        else atomicAdd(&counts[t], 1u);
    }
    bad = __reduce_add_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(err, (unsigned long long)bad);
}

// One block: exclusive scan of the tile counts into offsets[0 .. ntiles] and
// the scatter cursors.  Each thread scans a contiguous chunk.
__global__ void __launch_bounds__(1024) k_bin_scan(const unsigned *__restrict__ counts, int64_t ntiles,
                                                   int64_t *__restrict__ offsets,
                                                   unsigned long long *__restrict__ cursor) {
    __shared__ unsigned long long part[1024];
    const int64_t per = (ntiles + blockDim.x - 1) / blockDim.x;
    const int64_t b = threadIdx.x * per, e = min(ntiles, b + per);
    unsigned long long sum = 0;
    for (int64_t t = b; t < e; ++t) sum += counts[t];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int d = 1; d < (int)blockDim.x; d <<= 1) {  // inclusive Hillis-Steele scan of the chunk sums
        const unsigned long long v = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0ull;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = part[threadIdx.x] - sum;  // exclusive start of this chunk
    for (int64_t t = b; t < e; ++t) {
        offsets[t] = (int64_t)run;
        cursor[t] = run;
        run += counts[t];
    }
    if (threadIdx.x == blockDim.x - 1) offsets[ntiles] = (int64_t)part[threadIdx.x];
}

// The scatter writes each kept fragment as one record into its tile's next
// slot of a staging array -- 32 bytes (pixel, z, alpha, r, g, b) or 16 bytes
// (pixel, z, alpha) -- so that every slot is one whole-sector store, however
// scattered the slots are; a second pass copies the records out to the
// structure-of-arrays output in order, with coalesced loads and stores.
struct BinIn {
    const uint32_t *pixel;
    const float *z, *alpha, *r, *g, *b;
};
struct BinOut {
    uint32_t *pixel;
    float *z, *alpha, *r, *g, *b;
};

template <bool RGB>
__global__ void __launch_bounds__(256) k_bin_scatter(BinGeom g, int64_t n, BinIn a, uint4 *__restrict__ stage,
                                                     unsigned long long *__restrict__ cursor) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t px = a.pixel[i];
        const int64_t t = tile_index(px, g);
        if (t < 0) continue;
        const int64_t slot = (int64_t)atomicAdd(&cursor[t], 1ull);
        const uint4 r0 = make_uint4(px, __float_as_uint(a.z[i]), __float_as_uint(a.alpha[i]),
                                    RGB ? __float_as_uint(a.r[i]) : 0u);
        if (RGB) {
            stage[2 * slot] = r0;
            stage[2 * slot + 1] = make_uint4(__float_as_uint(a.g[i]), __float_as_uint(a.b[i]), 0u, 0u);
        } else {
            stage[slot] = r0;
        }
    }
}

template <bool RGB>
__global__ void __launch_bounds__(256) k_bin_unpack(int64_t n, const int64_t *__restrict__ kept_at,
                                                    const uint4 *__restrict__ stage, BinOut o) {
    const int64_t kept = *kept_at;  // tile_offsets[ntiles]
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < kept && i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 r0 = stage[RGB ? 2 * i : i];
        o.pixel[i] = r0.x;
        o.z[i] = __uint_as_float(r0.y);
        o.alpha[i] = __uint_as_float(r0.z);
        if (RGB) {
            const uint4 r1 = stage[2 * i + 1];
            o.r[i] = __uint_as_float(r0.w);
            o.g[i] = __uint_as_float(r1.x);
            o.b[i] = __uint_as_float(r1.y);
        }
    }
}

// Binning with per-block shared-memory counters, for descriptors whose tile
// count fits in shared memory: one block per SM owns a contiguous chunk of the
// stream.  Pass 1 counts the chunk's fragments per tile with shared atomics
// and stores the block's counts; a pass over the tiles turns them into each
// block's starting rank inside every tile (blocks in order) and the tile
// totals; pass 2 hands out ranks with shared atomics again, so no global
// atomic is issued per fragment.
constexpr int kBinThreads = 1024;

__global__ void __launch_bounds__(kBinThreads) k_bin_count_local(BinGeom g, int64_t n, int64_t chunk,
                                                                 int64_t ntiles, const uint32_t *__restrict__ pixel,
                                                                 unsigned *__restrict__ H, unsigned long long *err) {
    extern __shared__ unsigned hist[];
    for (int64_t t = threadIdx.x; t < ntiles; t += blockDim.x) hist[t] = 0u;
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * chunk, e = min(n, s + chunk);
    unsigned bad = 0;
    for (int64_t i = s + threadIdx.x; i < e; i += blockDim.x) {
        const int64_t t = tile_index(pixel[i], g);
        if (t < 0) ++bad;
        else atomicAdd(&hist[t], 1u);
    }
    bad = __reduce_add_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(err, (unsigned long long)bad);
    __syncthreads();
    unsigned *row = H + (int64_t)blockIdx.x * ntiles;
    for (int64_t t = threadIdx.x; t < ntiles; t += blockDim.x) row[t] = hist[t];
}

// Per tile: each block's count becomes the number of the tile's fragments in
// earlier blocks; the tile's total goes to counts[t].
__global__ void __launch_bounds__(256) k_bin_block_ranks(int nblocks, int64_t ntiles, unsigned *__restrict__ H,
                                                         unsigned *__restrict__ counts) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntiles) return;
    unsigned run = 0;
    for (int b = 0; b < nblocks; ++b) {
        const unsigned h = H[(int64_t)b * ntiles + t];
        H[(int64_t)b * ntiles + t] = run;
        run += h;
    }
    counts[t] = run;
}

template <bool RGB>
__global__ void __launch_bounds__(kBinThreads) k_bin_scatter_local(BinGeom g, int64_t n, int64_t chunk,
                                                                   int64_t ntiles, BinIn a,
                                                                   const unsigned *__restrict__ H,
                                                                   const int64_t *__restrict__ offsets,
                                                                   uint4 *__restrict__ stage) {
    extern __shared__ unsigned cur[];
    const unsigned *row = H + (int64_t)blockIdx.x * ntiles;
    for (int64_t t = threadIdx.x; t < ntiles; t += blockDim.x) cur[t] = row[t];
    __syncthreads();
    const int64_t s = (int64_t)blockIdx.x * chunk, e = min(n, s + chunk);
    for (int64_t i = s + threadIdx.x; i < e; i += blockDim.x) {
        const uint32_t px = a.pixel[i];
        const int64_t t = tile_index(px, g);
        if (t < 0) continue;
        const int64_t slot = offsets[t] + atomicAdd(&cur[t], 1u);
        const uint4 r0 = make_uint4(px, __float_as_uint(a.z[i]), __float_as_uint(a.alpha[i]),
                                    RGB ? __float_as_uint(a.r[i]) : 0u);
        if (RGB) {
            stage[2 * slot] = r0;
            stage[2 * slot + 1] = make_uint4(__float_as_uint(a.g[i]), __float_as_uint(a.b[i]), 0u, 0u);
        } else {
            stage[slot] = r0;
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
__global__ void __launch_bounds__(256) k_normalize_depth(int64_t n, int64_t P, const uint32_t *__restrict__ pixel,
                                                         const float *z, const float *__restrict__ zlo,
                                                         const float *__restrict__ zhi, float *z_out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t px = pixel[i];
        const float zi = z[i];
        float o = __int_as_float(0x7fc00000);
        if ((int64_t)px < P && zi == zi) {
            const float lo = zlo[px], range = zhi[px] - lo;
            o = range > 0.f && range < __int_as_float(0x7f800000) ? (zi - lo) / range : 0.f;
        }
        z_out[i] = o;
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
    g.width = d->width;
    g.height = d->height;
    g.tile_w = d->tile_w;
    g.tile_h = d->tile_h;
    g.ntx = (d->width + d->tile_w - 1) / d->tile_w;
    g.P = (int64_t)d->width * d->height;
    return g;
}

int64_t tiles_of(const wt_desc *d) {
    return (int64_t)((d->width + d->tile_w - 1) / d->tile_w) * ((d->height + d->tile_h - 1) / d->tile_h);
}

size_t ws_counts(int64_t ntiles) { return ((size_t)ntiles * 4 + 255) & ~size_t(255); }

int num_sms() {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// Tile counters that fit one block's shared memory (the per-block path).
bool local_bins(int64_t ntiles) { return ntiles * 4 <= 200 * 1024; }

// Bytes of the per-block count matrix (one row of ntiles per block).
size_t ws_blocks(int64_t ntiles) {
    return local_bins(ntiles) ? (((size_t)num_sms() * ntiles * 4 + 255) & ~size_t(255)) : 0;
}

}  // namespace
}  // namespace wt

using namespace wt;

extern "C" size_t wt_bin_workspace_bytes(const wt_desc *desc, int64_t n) {
    if (check_geom(desc) != WT_OK || n < 0) return 0;
    const int64_t nt = tiles_of(desc);
    return ws_counts(nt) + (((size_t)nt * 8 + 255) & ~size_t(255)) + ws_blocks(nt) + (size_t)n * 32;
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
    }
    unsigned long long *err = error_word();
    if (!err) return WT_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t nt = tiles_of(desc);
    char *ws = static_cast<char *>(workspace);
    unsigned *counts = reinterpret_cast<unsigned *>(ws);
    unsigned long long *cursor = reinterpret_cast<unsigned long long *>(ws + ws_counts(nt));
    const size_t blocks_bytes = ws_blocks(nt);
    unsigned *H = reinterpret_cast<unsigned *>(ws + ws_counts(nt) + (((size_t)nt * 8 + 255) & ~size_t(255)));
    uint4 *stage = reinterpret_cast<uint4 *>(reinterpret_cast<char *>(H) + blocks_bytes);
    const BinGeom g = bin_geom(desc);
    const BinIn a{in->pixel, in->z, in->alpha, in->r, in->g, in->b};
    const BinOut o{pixel_out, z_out, alpha_out, r_out, g_out, b_out};
    const int grid = grid_for(in->n);
    if (blocks_bytes && in->n > 0) {
        // per-block shared-memory counters
        const int nb = num_sms();
        const int64_t chunk = (in->n + nb - 1) / nb;
        const size_t smem = (size_t)nt * 4;
        cudaError_t e = cudaFuncSetAttribute(k_bin_count_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(rgb ? (const void *)k_bin_scatter_local<true> : (const void *)k_bin_scatter_local<false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return WT_ERR_CUDA;
        k_bin_count_local<<<nb, kBinThreads, smem, s>>>(g, in->n, chunk, nt, in->pixel, H, err);
        k_bin_block_ranks<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(nb, nt, H, counts);
        k_bin_scan<<<1, 1024, 0, s>>>(counts, nt, tile_offsets_out, cursor);
        if (rgb) {
            k_bin_scatter_local<true><<<nb, kBinThreads, smem, s>>>(g, in->n, chunk, nt, a, H, tile_offsets_out, stage);
            k_bin_unpack<true><<<grid, 256, 0, s>>>(in->n, tile_offsets_out + nt, stage, o);
        } else {
            k_bin_scatter_local<false><<<nb, kBinThreads, smem, s>>>(g, in->n, chunk, nt, a, H, tile_offsets_out, stage);
            k_bin_unpack<false><<<grid, 256, 0, s>>>(in->n, tile_offsets_out + nt, stage, o);
        }
        return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
    }
    // global atomics (tile counts too large for shared memory, or no fragments)
    if (cudaMemsetAsync(counts, 0, (size_t)nt * 4, s) != cudaSuccess) return WT_ERR_CUDA;
    if (in->n > 0) k_bin_count<<<grid, 256, 0, s>>>(g, in->n, in->pixel, counts, err);
    k_bin_scan<<<1, 1024, 0, s>>>(counts, nt, tile_offsets_out, cursor);
    if (in->n > 0) {
        if (rgb) {
            k_bin_scatter<true><<<grid, 256, 0, s>>>(g, in->n, a, stage, cursor);
            k_bin_unpack<true><<<grid, 256, 0, s>>>(in->n, tile_offsets_out + nt, stage, o);
        } else {
            k_bin_scatter<false><<<grid, 256, 0, s>>>(g, in->n, a, stage, cursor);
            k_bin_unpack<false><<<grid, 256, 0, s>>>(in->n, tile_offsets_out + nt, stage, o);
        }
    }
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
    k_normalize_depth<<<grid_for(frags->n), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        frags->n, (int64_t)desc->width * desc->height, frags->pixel, frags->z, zlo, zhi, z_out);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}
