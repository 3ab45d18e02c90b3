// band_static.cu -- nla_band2bd_noalloc: the band -> bidiagonal reduction for
// callers that cannot allocate device memory.
//
// nla_band2bd needs a small scratch array (one progress counter per group of
// sweeps of the bulge chase) that the caller normally supplies as a workspace.
// Some callers have no way to provide one: a plug-in or kernel library running
// inside a host framework whose memory manager owns the whole device and
// forbids allocations outside it, code that must never synchronise the device
// (cudaMalloc and cudaFree may), and programs with a fixed device-memory budget
// set at start-up.  For them this variant keeps its scratch in a fixed array
// compiled into the library.
//
// The array is a file-scope __device__ variable of kStaticChaseMaxN ints
// (256 KiB); every GPU that loads the library holds it until the process
// exits.  Host code cannot use the variable's name as a device address, so the
// first call on each device (with that device current) looks the address up
// with cudaGetSymbolAddress and caches it; make that first call before any
// stream capture.  All calls share the one array: the progress counters are
// cleared on the stream at the start of every call, and calls that overlap on
// the GPU (different streams without ordering between them) race on it and
// must not be issued.
#include <mutex>
#include <string>

#include "../../include/nla.h"
#include "common.cuh"
#include "kernels.cuh"
#include "trace.h"
#include "tuned.h"

namespace {

constexpr int kStaticChaseMaxN = 65536;  // largest n: one progress counter per sweep
constexpr int kMaxDevices = 64;

__device__ __align__(256) int g_chase_progress[kStaticChaseMaxN];

std::mutex g_mu;
int *g_progress_addr[kMaxDevices] = {};  // device address of g_chase_progress, per device

nla_status err(nla_status s, const char *msg) {
    nla_set_last_error(msg);
    return s;
}

}  // namespace

extern "C" nla_status nla_band2bd_noalloc(int n, int band, nla_dtype dtype, void *dAB, int ldab, double *dD,
                                          double *dE, int *dInfo, nla_stream_t stream) {
    if (dtype != NLA_F64 && dtype != NLA_F32) return err(NLA_ERR_ARG, "unknown dtype");
    if (n < 0 || band < 1 || band > 64) return err(NLA_ERR_ARG, "bad n or band");
    if (n > kStaticChaseMaxN)
        return err(NLA_ERR_UNSUPPORTED, "nla_band2bd_noalloc: n exceeds the static scratch limit of 65536");
    if (n == 0) return NLA_OK;
    if (!dAB || !dD || !dE || !dInfo) return err(NLA_ERR_ARG, "null device pointer");
    if (ldab < 3 * band + 1) return err(NLA_ERR_ARG, "ldab < 3*band+1");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return err(NLA_ERR_CUDA, "nla_band2bd_noalloc: no current CUDA device");
    }
    int *progress = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_progress_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_chase_progress);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return err(NLA_ERR_CUDA, "nla_band2bd_noalloc: cudaGetSymbolAddress failed");
            }
            g_progress_addr[dev] = static_cast<int *>(p);
        }
        progress = g_progress_addr[dev];
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(dInfo, 0, sizeof(int), st) != cudaSuccess) {
        cudaGetLastError();
        return err(NLA_ERR_CUDA, "nla_band2bd_noalloc: memset of info failed");
    }
    cudaError_t e;
    {
        nla::TraceScope ts(nla::kTrBand2bd, st);  // timed with the regular chase when tracing is on
        e = dtype == NLA_F64 ? nla::band2bd<double>((double *)dAB, ldab, n, band, dD, dE, progress, dInfo, st)
                             : nla::band2bd<float>((float *)dAB, ldab, n, band, dD, dE, progress, dInfo, st);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        std::string msg = std::string("nla_band2bd_noalloc: bulge chase: ") + cudaGetErrorString(e);
        return err(e == cudaErrorInvalidConfiguration ? NLA_ERR_CONFIG : NLA_ERR_CUDA, msg.c_str());
    }
    return NLA_OK;
}
