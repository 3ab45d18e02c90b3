// common.cuh -- small device/host helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "../../include/nla.h"

#define NLA_DEV __device__ __forceinline__

namespace nla {

// Device-side failure codes written to the caller's info word (negated status).
constexpr int kInfoTimeout = -NLA_ERR_TIMEOUT;

// Budget for every inter-block spin-wait, in nanoseconds of %globaltimer.
// A wait that exceeds it records kInfoTimeout and the kernel returns.
constexpr unsigned long long kSpinBudgetNs = 2000000000ull;  // 2 s

NLA_DEV unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

NLA_DEV unsigned int ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

NLA_DEV int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

NLA_DEV void st_release(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Spin until *p >= target or the budget runs out.  Called by one thread.
// Returns true on success; on timeout records kInfoTimeout in *info.  The
// sleep between polls doubles from 32 ns up to max_backoff_ns.
NLA_DEV bool spin_until_geq(const unsigned int *p, unsigned int target, int *info, unsigned max_backoff_ns = 256) {
    if (ld_acquire(p) >= target) return true;
    unsigned long long t0 = global_ns();
    unsigned int backoff = 32;
    while (true) {
        if (ld_acquire(p) >= target) return true;
        if (info && ld_acquire(info) == kInfoTimeout) return false;  // someone else gave up
        if (global_ns() - t0 > kSpinBudgetNs) {
            if (info) atomicExch(info, kInfoTimeout);
            return false;
        }
        __nanosleep(backoff);
        if (backoff < max_backoff_ns) backoff <<= 1;
    }
}

NLA_DEV bool spin_until_geq(const int *p, int target, int *info, unsigned max_backoff_ns = 256) {
    if (ld_acquire(p) >= target) return true;
    unsigned long long t0 = global_ns();
    unsigned int backoff = 32;
    while (true) {
        if (ld_acquire(p) >= target) return true;
        if (info && ld_acquire(info) == kInfoTimeout) return false;
        if (global_ns() - t0 > kSpinBudgetNs) {
            if (info) atomicExch(info, kInfoTimeout);
            return false;
        }
        __nanosleep(backoff);
        if (backoff < max_backoff_ns) backoff <<= 1;
    }
}

template <typename T>
NLA_DEV T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

NLA_DEV double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Loads that bypass L1 (data written by other blocks during the same launch).
NLA_DEV double ld_cg(const double *p) { return __ldcg(p); }
NLA_DEV float ld_cg(const float *p) { return __ldcg(p); }

// Programmatic dependent launch.  A kernel launched with launch_pdl may start while
// its predecessor in the stream is still running; pdl_wait() returns once the
// predecessor has completed and its memory operations are visible, so it comes
// before the kernel's first global-memory access.  pdl_trigger() lets the next
// kernel start launching (it will wait in its own pdl_wait()).  Both are no-ops
// for a kernel launched without the attribute.
NLA_DEV void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
NLA_DEV void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// NLA_PDL=1 adds the attribute (default: plain stream order).
bool pdl_enabled();

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

// ---------------------------------------------------------------- host: per-device set-up
// Launch set-up that depends on the device (a kernel's shared-memory or cluster
// attribute, an occupancy query, the SM count) is done once per device and may be
// reached from several host threads at the same time.

constexpr int kMaxDevices = 64;

// The current device (cudaGetDevice), or -1 when there is none.
int current_device();

// run(f) calls f() the first time it is reached while a given device is current and
// never again for that device; concurrent first calls wait for the one that runs f.
class PerDeviceOnce {
  public:
    template <class F>
    void run(F &&f) {
        const int dev = current_device();
        if (dev < 0 || dev >= kMaxDevices) {
            f();
            return;
        }
        const unsigned long long bit = 1ull << dev;
        if (done_.load(std::memory_order_acquire) & bit) return;
        std::lock_guard<std::mutex> lk(mu_);
        if (done_.load(std::memory_order_relaxed) & bit) return;
        f();
        done_.fetch_or(bit, std::memory_order_release);
    }

  private:
    std::atomic<unsigned long long> done_{0};
    std::mutex mu_;
};

// A value computed once per device (compute() runs with that device current).
template <class T>
class PerDeviceValue {
  public:
    template <class F>
    T get(F &&compute) {
        const int dev = current_device();
        if (dev < 0 || dev >= kMaxDevices) return compute();
        once_.run([&] { val_[dev] = compute(); });
        return val_[dev];
    }

  private:
    PerDeviceOnce once_;
    T val_[kMaxDevices] = {};
};

// Allow `kernel` the opt-in dynamic shared-memory maximum minus its static shared
// memory, once per device.
template <typename K>
void allow_max_smem(K kernel, PerDeviceOnce &once) {
    once.run([&] {
        int optin = 0;
        const int dev = current_device();
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev < 0 ? 0 : dev);
        cudaFuncAttributes fa;
        const size_t stat = cudaFuncGetAttributes(&fa, kernel) == cudaSuccess ? fa.sharedSizeBytes : 1024;
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)((size_t)optin - stat));
        cudaGetLastError();
    });
}

}  // namespace nla
