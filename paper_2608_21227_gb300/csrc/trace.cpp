// trace.cpp -- per-kernel-class CUDA-event timing (nla_trace_*).
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "../../include/nla.h"
#include "trace.h"

namespace {

const char *const kNames[nla::kTraceClasses] = {"panel_qr",     "panel_lq", "trail_left", "trail_right", "stage_copy",
                                                "band_extract", "band2bd",  "bisect",     "batched"};

struct Rec {
    int cls;
    cudaEvent_t a, b;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
int g_launch[nla::kTraceClasses] = {};
double g_ms[nla::kTraceClasses] = {};

cudaEvent_t take_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void drain_locked() {
    for (Rec &r : g_recs) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_launch[r.cls] += 1;
            g_ms[r.cls] += ms;
        }
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
}

}  // namespace

namespace nla {

bool trace_on() { return g_on; }

void *trace_begin(int cls, cudaStream_t st) {
    if (!g_on) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    Rec *r = new Rec{cls, take_event(), take_event()};
    cudaEventRecord(r->a, st);
    return r;
}

void trace_end(void *h, cudaStream_t st) {
    if (!h) return;
    Rec *r = static_cast<Rec *>(h);
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(r->b, st);
    g_recs.push_back(*r);
    delete r;
    if (g_recs.size() > 8192) drain_locked();  // bound the number of live events
}

}  // namespace nla

extern "C" {

nla_status nla_trace_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    return NLA_OK;
}

int nla_trace_read(nla_trace_entry *out, int max_entries) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    int k = 0;
    for (int c = 0; c < nla::kTraceClasses; ++c) {
        if (!g_launch[c]) continue;
        if (out && k < max_entries) out[k] = nla_trace_entry{kNames[c], g_launch[c], g_ms[c]};
        ++k;
    }
    return k;
}

void nla_trace_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    drain_locked();
    for (int c = 0; c < nla::kTraceClasses; ++c) {
        g_launch[c] = 0;
        g_ms[c] = 0.0;
    }
}

}  // extern "C"
