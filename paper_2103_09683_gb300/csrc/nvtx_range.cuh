// NVTX ranges around the C ABI's calls, named after them, so that a profiler's
// timeline shows which library call launched which kernels.  NVTX v3 is header
// only: with no profiler attached a range costs one branch on a null hook.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace dose {

class NvtxRange {
  public:
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace dose
