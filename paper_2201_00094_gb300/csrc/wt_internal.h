// Internal interface between the C-ABI layer (wt_api.cu) and the per-dtype
// kernel translation units.  Not installed; not part of the ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace wt {

struct Params;

// One entry of a serving step's task table: a slot (admitted frame) and a
// range of its tiles; start is the running sum of range lengths before it.
struct ServeTask {
    int32_t slot;
    int32_t tile0;
    int64_t start;
};

typedef cudaError_t (*TileLaunch)(const Params &, int ntiles, cudaStream_t);
typedef cudaError_t (*ServeLaunch)(const Params *slots, const ServeTask *tasks, int ntasks,
                                   int64_t total, unsigned long long *counter, int npx, int grid,
                                   cudaStream_t);
typedef int (*ServeOccupancy)(int npx);
typedef cudaError_t (*TemporalLaunch)(const Params &, int ntiles, const void *coeff_prev, const float *zmin_prev,
                                      cudaStream_t);
typedef cudaError_t (*QueryLaunch)(const Params &, int64_t q, const uint32_t *qpx, const float *qz,
                                   const float *qal, float *outA, cudaStream_t);

// [J-1] for J = 1..5; suffix = storage type (0 f32, 1 bf16, 2 f16)
extern const TileLaunch kBuild0[5], kBuild1[5], kBuild2[5];
extern const TileLaunch kResolve0[5], kResolve1[5], kResolve2[5];
extern const TileLaunch kResolveComp0[5], kResolveComp1[5], kResolveComp2[5];
extern const TileLaunch kFused0[5], kFused1[5], kFused2[5];
extern const TileLaunch kBackward0[5], kBackward1[5], kBackward2[5];
extern const ServeLaunch kServe0[5], kServe1[5], kServe2[5];
extern const ServeOccupancy kServeOcc0[5], kServeOcc1[5], kServeOcc2[5];
extern const QueryLaunch kAbsorbance0[5], kAbsorbance1[5], kAbsorbance2[5];
extern const TemporalLaunch kTemporal0[5], kTemporal1[5], kTemporal2[5];

// Coloured absorbance (wt_rgb.cu): shared memory of a tile, and the launch.
size_t rgb_smem_bytes(int J, int npx, bool e5);
cudaError_t launch_fused_rgb(const Params &p, int J, const float *const alpha_c[3], bool e5, int ntiles,
                             cudaStream_t s);

}  // namespace wt
