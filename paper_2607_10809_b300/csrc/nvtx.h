// NVTX range over a scope for the host entry points of the C ABI (not part of
// the public interface).
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace hw {

// Names the host-side phases (mesh precompute, state upload, steps, runs,
// adjoint steps, batches) on a profiler timeline; it costs nothing when no
// tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace hw
