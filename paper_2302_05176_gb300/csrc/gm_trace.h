// gm_trace.h -- NVTX ranges around the library's host entry points, so that a
// timeline profiler shows each call (and each serving batch, each host-pipeline
// chunk) by name.  NVTX is header-only; without an attached tool a range costs a
// function-pointer check.
#pragma once
#include <nvtx3/nvToolsExt.h>

namespace gm {

struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace gm
