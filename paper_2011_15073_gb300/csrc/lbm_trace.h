// lbm_trace.h -- NVTX ranges around the library's host entry points, so that
// a timeline (Nsight Systems) shows steps, reductions, sweeps and the
// adjoint by name.  NVTX v3 is header-only: without a tool attached each
// range is a check of a null function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace lbm {
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};
}  // namespace lbm

#define LBM_TRACE(name) lbm::TraceRange lbm_trace_range_(name)
