// NVTX ranges around the host entry points and serving ticks, so a profiler
// timeline shows the solver's phases (header-only NVTX; no cost without a
// tool attached).
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace admm_impl {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

} // namespace admm_impl
