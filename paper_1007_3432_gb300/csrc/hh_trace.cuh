// NVTX ranges over the host-side phases of the library's calls (solve,
// trajectory stages, applies, batch chunks, slab halo exchanges), so that a
// timeline profiler shows which call enqueued which kernels.  NVTX v3 is
// header-only: without a profiler attached a range costs one indirect call.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace hh {

struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

}  // namespace hh
