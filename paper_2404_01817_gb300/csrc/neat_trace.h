// NVTX ranges around the library's host entry points (NVTX3, header only):
// with no profiler attached a range costs a check of a function pointer;
// under Nsight tools (or ncu --nvtx --nvtx-include) the ranges name and
// delimit each call's launches.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace neat {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace neat
