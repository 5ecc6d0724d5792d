// NVTX ranges around the library's host-side phases (set-up, the run's graph capture and replay,
// autotuning, state and result transfers, checkpoints, the stateless calls), so that a timeline
// or an `ncu --nvtx --nvtx-include` filter can attribute kernels to them.  NVTX3 is header-only
// and costs a few nanoseconds per range when no tool is attached.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace nefe {

struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace nefe
