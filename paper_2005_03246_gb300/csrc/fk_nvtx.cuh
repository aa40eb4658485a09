// fk_nvtx.cuh -- NVTX ranges around the library's entry points, so that a
// timeline tool (Nsight Systems, or ncu's --nvtx filters) shows each call as
// one named range over the kernels it launches.  The NVTX v3 header is
// header-only; with no tool attached a range costs one indirect call.  Where
// the toolkit has no NVTX headers the ranges compile to nothing.
#pragma once

#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define FK_HAVE_NVTX 1
#endif
#endif

namespace fk {
struct NvtxRange {
    explicit NvtxRange(const char* name) {
#ifdef FK_HAVE_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~NvtxRange() {
#ifdef FK_HAVE_NVTX
        nvtxRangePop();
#endif
    }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace fk

#define FK_RANGE(name) ::fk::NvtxRange fk_nvtx_range_(name)
