// NVTX ranges around the library's host entry points, so that a solve, an
// autotuning run or a server step shows up as one named span in Nsight
// timelines and can be selected with ncu --nvtx.  NVTX3 is header-only; with
// no tool attached a range costs a branch.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace fabm {

class TraceRange {
public:
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace fabm
