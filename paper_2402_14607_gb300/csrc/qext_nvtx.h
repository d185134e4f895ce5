// NVTX ranges around the host-side stages of the entry points (ingest,
// extraction, host<->device copies, batches, serving rounds), so that a
// timeline tool shows where each call spends its time.  NVTX v3 is header
// only; with no tool attached a range costs a check of a function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace qext {

// One named range for the lifetime of the object (push on construction,
// pop on destruction).
class NvtxRange {
   public:
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace qext
