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

// Largest J (Haar levels) of the mono kernels; 64 coefficients per pixel.
constexpr int kMaxJ = 6;
// Shared memory one CTA may use on sm_103a; a layout beyond it is refused
// (the launchers return cudaErrorNotSupported, reported as WT_ERR_UNSUPPORTED).
constexpr size_t kMaxSmemPerBlock = 227 * 1024;

// [J-1] for J = 1..kMaxJ; suffix = storage type (0 f32, 1 bf16, 2 f16, 3 shared-exponent 16-bit)
extern const TileLaunch kBuild0[kMaxJ], kBuild1[kMaxJ], kBuild2[kMaxJ], kBuild3[kMaxJ];
extern const TileLaunch kResolve0[kMaxJ], kResolve1[kMaxJ], kResolve2[kMaxJ], kResolve3[kMaxJ];
extern const TileLaunch kResolveComp0[kMaxJ], kResolveComp1[kMaxJ], kResolveComp2[kMaxJ], kResolveComp3[kMaxJ];
extern const TileLaunch kFused0[kMaxJ], kFused1[kMaxJ], kFused2[kMaxJ], kFused3[kMaxJ];
extern const TileLaunch kBackward0[kMaxJ], kBackward1[kMaxJ], kBackward2[kMaxJ], kBackward3[kMaxJ];
extern const ServeLaunch kServe0[kMaxJ], kServe1[kMaxJ], kServe2[kMaxJ], kServe3[kMaxJ];
extern const ServeOccupancy kServeOcc0[kMaxJ], kServeOcc1[kMaxJ], kServeOcc2[kMaxJ], kServeOcc3[kMaxJ];
extern const QueryLaunch kAbsorbance0[kMaxJ], kAbsorbance1[kMaxJ], kAbsorbance2[kMaxJ], kAbsorbance3[kMaxJ];
extern const TemporalLaunch kTemporal0[kMaxJ], kTemporal1[kMaxJ], kTemporal2[kMaxJ], kTemporal3[kMaxJ];

// The table of a storage type (0..3 as above); t[dtype].
template <typename T> inline const T *by_dtype(int32_t dt, const T *t0, const T *t1, const T *t2, const T *t3) {
    return dt == 0 ? t0 : dt == 1 ? t1 : dt == 2 ? t2 : t3;
}

// Bytes of one frame's coefficient storage: P * 2^J stored values, plus one
// exponent byte per pixel for the shared-exponent type; 0 for an unknown type.
inline size_t coeff_storage_bytes(int64_t P, int J, int32_t dt) {
    const size_t C = (size_t)1 << J;
    switch (dt) {
    case 0: return (size_t)P * C * 4;
    case 1:
    case 2: return (size_t)P * C * 2;
    case 3: return (size_t)P * C * 2 + (size_t)P;
    default: return 0;
    }
}

// Coloured absorbance (wt_rgb.cu): shared memory of a tile, and the launch.
size_t rgb_smem_bytes(int J, int npx, bool e5);
cudaError_t launch_fused_rgb(const Params &p, int J, const float *const alpha_c[3], bool e5, int ntiles,
                             cudaStream_t s);

}  // namespace wt
