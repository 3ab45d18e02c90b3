// trace.h -- internal hooks of the per-kernel-class timing (nla_trace_*).
#pragma once
#include <cuda_runtime.h>

namespace nla {

enum TraceClass {
    kTrPanelQR = 0,
    kTrPanelLQ,
    kTrTrailLeft,
    kTrTrailRight,
    kTrStageCopy,
    kTrBandExtract,
    kTrBand2bd,
    kTrBisect,
    kTrBatched,
    kTraceClasses
};

bool trace_on();
void *trace_begin(int cls, cudaStream_t st);
void trace_end(void *h, cudaStream_t st);

// Brackets one launch: NLA_TRACED(class, stream, expression returning cudaError_t).
struct TraceScope {
    void *h;
    cudaStream_t st;
    TraceScope(int cls, cudaStream_t s) : h(trace_on() ? trace_begin(cls, s) : nullptr), st(s) {}
    ~TraceScope() { trace_end(h, st); }
};

}  // namespace nla
