// rsc_trace.h -- NVTX ranges of the library's entry points.
#pragma once

#include <nvtx3/nvToolsExt.h>

// NVTX range over a scope: a tracing tool (Nsight Systems, ncu --nvtx) shows
// the library's calls and the FP16 path's stream groups by name; without a
// tool attached the calls return at once.
struct RscRange {
  explicit RscRange(const char *name) { nvtxRangePushA(name); }
  ~RscRange() { nvtxRangePop(); }
  RscRange(const RscRange &) = delete;
  RscRange &operator=(const RscRange &) = delete;
};
