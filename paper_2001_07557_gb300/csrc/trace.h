// trace.h -- NVTX ranges around the library's entry points and solver phases,
// for timelines and for range-filtered profiling, e.g.
//   ncu --nvtx --nvtx-include "lqcd/cg/inner/" ...
// Range names are "lqcd/<call>" and "lqcd/cg/<phase>".  NVTX v3 is header-only:
// with no tool attached, a range costs one indirect call that returns at once.
// The ranges mark host-side calls; inside a captured CUDA graph they mark the
// capture, not the replays.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace lq {

struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace lq
