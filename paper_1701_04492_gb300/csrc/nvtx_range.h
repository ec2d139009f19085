// nvtx_range.h -- an NVTX range around each C-ABI call (plan, exec, inverse), so that
// a profiler's timeline shows the library's stages.  NVTX3 is header-only; without
// a tool attached a range costs a check of one function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace nufft {
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace nufft
