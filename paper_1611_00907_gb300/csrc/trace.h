// NVTX ranges around the library's entry points, so that Nsight Systems and
// Nsight Compute (`ncu --nvtx --nvtx-include "lbm_step/"`) place the
// kernels under the call that launched them.  NVTX v3 is header-only; with
// no tool attached a range costs a few nanoseconds.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace cplbm {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace cplbm

// A range named `name` from here to the end of the enclosing scope.
#define CPLBM_TRACE(name) ::cplbm::TraceRange cplbm_trace_range_(name)
