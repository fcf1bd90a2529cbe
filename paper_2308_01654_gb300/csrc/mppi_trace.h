// mppi_trace.h - the library's NVTX ranges (domain "mppi"): one around each kernel launch of an
// iteration and one per serving micro-batch from its submission to its completion.  Nsight
// Systems and Nsight Compute (--nvtx) show them; without an attached tool each call returns at
// once.
#pragma once

#include <nvtx3/nvToolsExt.h>

namespace mppi {

inline nvtxDomainHandle_t trace_domain() {
    static nvtxDomainHandle_t d = nvtxDomainCreateA("mppi");
    return d;
}

inline nvtxEventAttributes_t trace_attr(const char* name) {
    nvtxEventAttributes_t a{};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = name;
    return a;
}

// A range for the enclosing scope on the calling thread.
struct TraceScope {
    explicit TraceScope(const char* name) {
        const nvtxEventAttributes_t a = trace_attr(name);
        nvtxDomainRangePushEx(trace_domain(), &a);
    }
    ~TraceScope() { nvtxDomainRangePop(trace_domain()); }
    TraceScope(const TraceScope&) = delete;
    TraceScope& operator=(const TraceScope&) = delete;
};

// A range that may end on another thread (a micro-batch: submitted by the scheduler, completed
// by the completion thread).
inline nvtxRangeId_t trace_start(const char* name) {
    const nvtxEventAttributes_t a = trace_attr(name);
    return nvtxDomainRangeStartEx(trace_domain(), &a);
}

inline void trace_end(nvtxRangeId_t id) { nvtxDomainRangeEnd(trace_domain(), id); }

}  // namespace mppi
