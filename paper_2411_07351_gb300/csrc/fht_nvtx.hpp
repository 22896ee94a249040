// NVTX ranges around the host-side enqueue of each kernel launch, so that a
// timeline (nsys or any NVTX-aware tool) names every pass of the transform.
// Without a tool attached a range costs a pointer test.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace fht {

struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace fht
