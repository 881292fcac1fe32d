/*
 * NVTX ranges around the engine's host entry points that launch device work, so that a
 * profiler's timeline groups the launches and `ncu --nvtx --nvtx-include "<range>/"`
 * captures one of them.  NVTX3 is header-only: with no tool attached a range costs a
 * pointer check.  Without the header the ranges compile to nothing.
 */
#ifndef GX_TRACE_H
#define GX_TRACE_H

#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define GX_HAVE_NVTX 1
#endif
#endif

namespace gx {

/* a range open for the lifetime of the object (one per scope, on the calling thread) */
struct TraceRange {
    explicit TraceRange(const char *name) {
#ifdef GX_HAVE_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~TraceRange() {
#ifdef GX_HAVE_NVTX
        nvtxRangePop();
#endif
    }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

} // namespace gx

#endif
