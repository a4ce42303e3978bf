// NVTX ranges around the host-side phases of the library (a Parareal run, its coarse initial
// sweep, each iteration's fine and coarse sweeps, the sequential reference, propagations, G_theta
// training and inference), so that a profiler can attribute kernels to the phase that launched
// them (for example `ncu --nvtx --nvtx-include "fine sweep/"`). NVTX v3 is header-only: without a
// tool attached each push and pop is one call that returns at once. Where the toolkit has no NVTX
// headers the ranges compile to nothing.
#pragma once

#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define CH_HAVE_NVTX 1
#endif
#endif

namespace chtrace {

// A range open for the lifetime of the object (nested ranges stack).
class Range {
 public:
  explicit Range(const char* name) {
#ifdef CH_HAVE_NVTX
    nvtxRangePushA(name);
#else
    (void)name;
#endif
  }
  ~Range() {
#ifdef CH_HAVE_NVTX
    nvtxRangePop();
#endif
  }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

}  // namespace chtrace
