// NVTX ranges around the library's entry points and their phases, in the
// NVTX domain "hc": Nsight tools (and any NVTX injection library) see them;
// with no tool attached a range costs a few nanoseconds.  Host-side ranges:
// they mark when the work was enqueued, the tools map them onto the GPU.
#pragma once

#include <cstring>

#include <nvtx3/nvToolsExt.h>

namespace hc {

inline nvtxDomainHandle_t trace_domain() {
    static const nvtxDomainHandle_t d = nvtxDomainCreateA("hc");
    return d;
}

// A range for the lifetime of the object (one scope).
class TraceRange {
  public:
    explicit TraceRange(const char* name) {
        nvtxEventAttributes_t a;
        std::memset(&a, 0, sizeof(a));
        a.version = NVTX_VERSION;
        a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
        a.messageType = NVTX_MESSAGE_TYPE_ASCII;
        a.message.ascii = name;
        nvtxDomainRangePushEx(trace_domain(), &a);
    }
    ~TraceRange() { nvtxDomainRangePop(trace_domain()); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};

}  // namespace hc
