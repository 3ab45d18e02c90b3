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

// ---- pipe microbenchmarks: long chains of independent FMAs / tensor-core MMAs

template <typename T>
__global__ void __launch_bounds__(256) fma_pipe_kernel(int iters, T seed, T *out) {
    constexpr int kChains = 8;  // independent accumulators per thread hide the FMA latency
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = seed + (T)(threadIdx.x + c);
    const T x = (T)0.999999, y = (T)1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = a[c] * x + y;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == (T)-1) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // never true: keeps the chains alive
}

// One block per SM: one thread issues `iters` kind::tf32 MMAs (M = 128, N = 256, K = 8)
// on fixed shared-memory operands into a TMEM accumulator, then waits (bounded) for them.
__global__ void __launch_bounds__(128) tf32_pipe_kernel(int iters, float *out, int *info) {
    __shared__ __align__(1024) unsigned char ops[128 * 32 + 256 * 32];
    __shared__ __align__(8) uint64_t done;
    __shared__ uint32_t tbase_sh;
    const int tid = threadIdx.x, warp = tid >> 5;
    for (int i = tid; i < (128 + 256) * 8; i += blockDim.x)
        reinterpret_cast<uint32_t *>(ops)[i] = tc::to_tf32(1.0f + 1e-3f * (float)(i & 15));
    if (warp == 0) {
        tc::tmem_alloc(&tbase_sh, 256);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = tbase_sh;
    if (tid == 0) {
        const uint64_t a = tc::sdesc(tc::smem_u32(ops), 128, 8 * 32);
        const uint64_t b = tc::sdesc(tc::smem_u32(ops + 128 * 32), 128, 8 * 32);
        const uint32_t id = tc::idesc(2, 128, 256);
        for (int i = 0; i < iters; ++i) tc::mma_tf32(tb, a, b, id, i > 0 ? 1u : 0u);
        tc::mma_commit(&done);
    }
    const bool ok = tc::mbar_wait_warp(&done, 0, info);
    tc::fence_after_sync();
    if (ok && warp == 0) {
        float v[16];
        tc::tmem_ld16(tb, v);
        tc::tmem_wait_ld();
        if (v[0] == -1.f) out[blockIdx.x] = v[1];  // never true
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tb, 256);
}

}  // namespace
}  // namespace nla

extern "C" nla_status nla_pipe_selftest(int kind, int blocks, int iters, void *dOut, int *dInfo,
                                        nla_stream_t stream) {
    if (kind < 0 || kind > 2 || blocks < 1 || blocks > 65536 || iters < 1 || !dOut || !dInfo) return NLA_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (kind == 0)
        nla::fma_pipe_kernel<float><<<blocks, 256, 0, st>>>(iters, 0.5f, (float *)dOut);
    else if (kind == 1)
        nla::fma_pipe_kernel<double><<<blocks, 256, 0, st>>>(iters, 0.5, (double *)dOut);
    else
        nla::tf32_pipe_kernel<<<blocks, 128, 0, st>>>(iters, (float *)dOut, dInfo);
    return cudaGetLastError() == cudaSuccess ? NLA_OK : NLA_ERR_CUDA;
}

extern "C" nla_status nla_wait_selftest(int mode, int budget_us, int *dInfo, nla_stream_t stream) {
    if ((mode != 0 && mode != 1) || budget_us < 1 || budget_us > 2000000 || !dInfo) return NLA_ERR_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    nla::wait_selftest_kernel<<<1, 32, 0, st>>>(mode, (unsigned long long)budget_us * 1000ull, dInfo);
    return cudaGetLastError() == cudaSuccess ? NLA_OK : NLA_ERR_CUDA;
}
