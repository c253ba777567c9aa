// wt_build_resolve_batch_static: a batch of frames through one persistent
// launch of the fused kernel, with every piece of device scratch it needs
// taken from a small array that is part of the library image.
//
// Some callers cannot allocate device memory at the point where they submit
// a frame: a renderer that reserves its whole device budget at start-up and
// must not grow it afterwards (for example when the GPU's memory is split
// between processes), or a real-time loop in which a cudaMalloc / cudaFree --
// which can synchronise the whole device -- would stall other work in flight.
// This entry point lets them batch frames without any allocation: the
// per-frame parameter table, the tile-range table and the work counter live
// in the statically sized array below.  Inputs and outputs are the caller's.
#include <cstddef>
#include <cstring>
#include <mutex>

#include "wt.h"
#include "wt_internal.h"
#include "wt_trace.h"
#include "wt_tile.cuh"

namespace wt {
namespace {

constexpr int kStaticBatchFrames = 64;  // frames per call (the stated maximum)

// Layout of the scratch: the work counter on its own 256-byte line, then one
// parameter block and one tile range per frame.
struct StaticBatch {
    unsigned long long counter;
    unsigned long long pad[31];
    Params params[kStaticBatchFrames];
    ServeTask tasks[kStaticBatchFrames];
};

// The scratch itself: part of the library's device image, so every GPU that
// loads the library holds these bytes until the process exits.  In host code
// this name is only a host-side stand-in for the symbol; the device address
// comes from cudaGetSymbolAddress (below).
static __device__ __align__(256) unsigned char g_batch_scratch[sizeof(StaticBatch)];

constexpr int kMaxDevices = 64;
StaticBatch *g_scratch_ptr[kMaxDevices];
cudaError_t g_scratch_status[kMaxDevices];
std::once_flag g_scratch_once[kMaxDevices];

// Device address of the scratch on the current device, resolved once per
// device with that device current.
StaticBatch *scratch_address(int dev) {
    std::call_once(g_scratch_once[dev], [dev] {
        void *ptr = nullptr;
        g_scratch_status[dev] = cudaGetSymbolAddress(&ptr, g_batch_scratch);
        if (g_scratch_status[dev] == cudaSuccess) g_scratch_ptr[dev] = static_cast<StaticBatch *>(ptr);
    });
    return g_scratch_ptr[dev];
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

unsigned long long *error_word();  // wt_api.cu

}  // namespace wt

using namespace wt;

extern "C" wt_status wt_build_resolve_batch_static(const wt_desc *descs, const wt_frags *frags,
                                                   const float *bgs, float *const *outs,
                                                   int32_t nframes, wt_stream stream) {
    WT_TRACE();
    if (!descs || !frags || !bgs || !outs) return WT_ERR_ARG;
    if (nframes < 1 || nframes > kStaticBatchFrames) return WT_ERR_ARG;  // beyond the stated maximum
    const wt_desc &d0 = descs[0];
    if (d0.J < 1 || d0.J > 5) return d0.J < 1 ? WT_ERR_ARG : WT_ERR_UNSUPPORTED;
    if (d0.coeff_dtype != WT_F32 && d0.coeff_dtype != WT_BF16 && d0.coeff_dtype != WT_F16) return WT_ERR_ARG;
    if (d0.tile_w < 1 || d0.tile_h < 1 || (int64_t)d0.tile_w * d0.tile_h > kMaxTilePx) return WT_ERR_ARG;

    // host staging on the stack: no heap or device allocation anywhere
    StaticBatch host;
    host.counter = 0;  // the claim counter must start at zero on every call
    for (int i = 0; i < 31; ++i) host.pad[i] = 0;
    int64_t total = 0;
    unsigned long long *err = error_word();
    if (!err) return WT_ERR_CUDA;
    for (int k = 0; k < nframes; ++k) {
        const wt_desc &d = descs[k];
        const wt_frags &f = frags[k];
        // one kernel instantiation and one shared-memory layout per launch
        if (d.J != d0.J || d.coeff_dtype != d0.coeff_dtype || d.tile_w != d0.tile_w || d.tile_h != d0.tile_h)
            return WT_ERR_UNSUPPORTED;
        if (d.width < 1 || d.height < 1 || (int64_t)d.width * d.height >= (int64_t(1) << 31) || d.reserved)
            return WT_ERR_ARG;
        if (d.flags & ~uint32_t(WT_SELF_EXCLUDE | WT_INTERP_LINEAR | WT_RESOLVE_NORMALIZED)) return WT_ERR_ARG;
        if (f.n < 0 || !f.tile_offsets || !outs[k] || !aligned16(outs[k])) return WT_ERR_ARG;
        const void *req[6] = {f.pixel, f.z, f.alpha, f.r, f.g, f.b};
        for (const void *p : req)
            if ((f.n > 0 && !p) || !aligned16(p)) return WT_ERR_ARG;
        Params &p = host.params[k];
        memset(&p, 0, sizeof(p));
        p.g.width = d.width;
        p.g.height = d.height;
        p.g.tile_w = d.tile_w;
        p.g.tile_h = d.tile_h;
        p.g.ntx = (d.width + d.tile_w - 1) / d.tile_w;
        p.flags = d.flags;
        set_row_division(p);
        p.n = f.n;
        p.pixel = f.pixel;
        p.z = f.z;
        p.alpha = f.alpha;
        p.r = f.r;
        p.gc = f.g;
        p.b = f.b;
        p.off = f.tile_offsets;
        p.out = outs[k];
        p.bg0 = bgs[3 * k];
        p.bg1 = bgs[3 * k + 1];
        p.bg2 = bgs[3 * k + 2];
        p.err = err;
        const int64_t tiles = (int64_t)p.g.ntx * ((d.height + d.tile_h - 1) / d.tile_h);
        host.tasks[k].slot = k;
        host.tasks[k].tile0 = 0;
        host.tasks[k].start = total;
        total += tiles;
    }

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return WT_ERR_CUDA;
    StaticBatch *scratch = scratch_address(dev);
    if (!scratch) return WT_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return WT_ERR_CUDA;
    const int dt = d0.coeff_dtype;
    const ServeOccupancy *O = dt == WT_F32 ? kServeOcc0 : (dt == WT_BF16 ? kServeOcc1 : kServeOcc2);
    const ServeLaunch *L = dt == WT_F32 ? kServe0 : (dt == WT_BF16 ? kServe1 : kServe2);
    const int npx = d0.tile_w * d0.tile_h;
    const int occ = O[d0.J - 1](npx);
    if (occ < 1) return WT_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the counter (zeroed above) and the tables of this call; a copy from
    // pageable host memory is staged by the runtime before the call returns
    char *base = reinterpret_cast<char *>(scratch);
    const size_t params_off = offsetof(StaticBatch, params);
    const size_t tasks_off = offsetof(StaticBatch, tasks);
    if (cudaMemcpyAsync(base, &host, params_off, cudaMemcpyHostToDevice, s) != cudaSuccess) return WT_ERR_CUDA;
    if (cudaMemcpyAsync(base + params_off, &host.params[0], sizeof(Params) * nframes,
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        return WT_ERR_CUDA;
    if (cudaMemcpyAsync(base + tasks_off, &host.tasks[0], sizeof(ServeTask) * nframes,
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        return WT_ERR_CUDA;
    if (total == 0) return WT_OK;
    const int grid = (int)(total < (int64_t)sms * occ ? total : (int64_t)sms * occ);
    const cudaError_t e =
        L[d0.J - 1](reinterpret_cast<const Params *>(base + params_off),
                    reinterpret_cast<const ServeTask *>(base + tasks_off), nframes, total,
                    reinterpret_cast<unsigned long long *>(base), npx, grid, s);
    return e == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}
