// diag.cu -- failure-detection self-test: bounded waits that run out.
//
// Every inter-block or inter-warp wait of the library is bounded: a spin on a
// global counter (cooperative panel, bulge chase, batched queue) or an
// mbarrier wait (TMA / tensor-core pipelines) gives up after a time budget,
// records -NLA_ERR_TIMEOUT in the caller's info word and returns.  This kernel
// exercises both forms on a condition that never becomes true, with a short
// budget, so that a test can check the status and that the context survives.
#include "../../include/nla.h"
#include "common.cuh"
#include "tc.cuh"

namespace nla {
namespace {

__device__ unsigned int g_never;  // zero-initialised; nothing ever writes it

__global__ void wait_selftest_kernel(int mode, unsigned long long budget_ns, int *info) {
    unsigned int *never = &g_never;
    __shared__ __align__(8) uint64_t mbar;
    if (threadIdx.x != 0) return;
    bool ok = true;
    if (mode == 0) {
        const unsigned long long t0 = global_ns();
        ok = false;
        unsigned ns = 32;
        while (global_ns() - t0 <= budget_ns) {
            if (ld_acquire(never) >= 1u) {
                ok = true;
                break;
            }
            __nanosleep(ns);
            if (ns < 1024) ns <<= 1;
        }
    } else {
        tc::mbar_init(&mbar, 1);  // one arrival expected; none comes
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const unsigned long long t0 = global_ns();
        ok = false;
        while (global_ns() - t0 <= budget_ns) {
            if (tc::mbar_try_wait(&mbar, 0)) {
                ok = true;
                break;
            }
        }
    }
    if (!ok) atomicExch(info, kInfoTimeout);
}

}  // namespace
}  // namespace nla

extern "C" nla_status nla_wait_selftest(int mode, int budget_us, int *dInfo, nla_stream_t stream) {
    if ((mode != 0 && mode != 1) || budget_us < 1 || budget_us > 2000000 || !dInfo) return NLA_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    nla::wait_selftest_kernel<<<1, 32, 0, st>>>(mode, (unsigned long long)budget_us * 1000ull, dInfo);
    return cudaGetLastError() == cudaSuccess ? NLA_OK : NLA_ERR_CUDA;
}
