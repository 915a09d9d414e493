// vegas_nvtx.h -- one NVTX range per public C-ABI call, so that a profiler
// (ncu --nvtx, Nsight Systems) can attribute kernels and copies to the call
// that issued them.  NVTX v3 is header-only: without an attached tool every
// push and pop is a call through a null-initialised pointer that returns at
// once.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace vegas {

struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace vegas

// A range named after the enclosing C-ABI function, open until it returns.
#define VEGAS_NVTX_RANGE() const ::vegas::NvtxRange vegas_nvtx_range_(__func__)
