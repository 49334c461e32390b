// qs_nvtx.h -- NVTX ranges around the library's entry points, so that a
// profiler (ncu --nvtx, Nsight Systems) attributes every kernel to the call
// that enqueued it.  NVTX 3 is header-only: with no tool attached a range
// costs one check of a function pointer.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace qsp {
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
}  // namespace qsp

#define QS_RANGE(name) const qsp::NvtxRange qs_nvtx_range_(name)
