// NVTX ranges over the C-ABI calls (header-only NVTX: a no-op unless a
// profiler is attached), so that traces show each call of the library by name.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace wt {
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace wt

#define WT_TRACE() ::wt::NvtxRange wt_trace_range_(__func__)
