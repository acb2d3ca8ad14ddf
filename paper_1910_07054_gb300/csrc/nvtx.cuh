// NVTX ranges around the host-side stages (plan build, row transforms,
// columns and layer sum), so that a profiler attached to the process shows
// and can filter them.  NVTX 3 is header-only and costs nothing without an
// attached tool; where the toolkit lacks its header the ranges compile away.
#pragma once

#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define DEMAG_HAVE_NVTX 1
#endif
#endif

namespace demag {

struct NvtxRange {
    explicit NvtxRange(const char *name) {
#ifdef DEMAG_HAVE_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~NvtxRange() {
#ifdef DEMAG_HAVE_NVTX
        nvtxRangePop();
#endif
    }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

}  // namespace demag
