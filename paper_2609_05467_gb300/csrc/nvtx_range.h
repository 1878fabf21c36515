// nvtx_range.h -- an NVTX range around each library call, so that a
// timeline tool (Nsight Systems, Nsight Compute's NVTX filters) shows which
// call a kernel belongs to.  NVTX is header-only and does nothing when no
// tool is attached.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace rc {

struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace rc

#define RC_RANGE() ::rc::NvtxRange rc_nvtx_range_(__func__)
