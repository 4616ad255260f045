// NVTX ranges around the library's host entry points (steps, batch runs, serving chunks, transfers),
// so that a profiler's timeline shows which call issued which launches.  NVTX v3 is header-only: with
// no tool attached a range costs a branch on an unset function pointer.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace assn {

struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace assn
