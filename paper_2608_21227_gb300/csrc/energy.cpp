// energy.cpp -- the tuner's energy observer (paper Section 3.1 and Section 6: tuning
// for energy through observers of the device's power/energy counters).
//
// NVML is opened at run time (dlopen of libnvidia-ml.so.1, or the library named by
// NLA_NVML_LIB), so the library neither links nor requires it.  Only read-only queries
// are made: the device's total energy counter (millijoules since the driver loaded).
// Nothing here changes any setting of the GPU.
#include <dlfcn.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/kt.h"
#include "../../include/nla.h"
#include "tuned.h"

namespace {

typedef struct nvml_device_st *nvml_device;  // opaque NVML handle
typedef int (*fn_init)(void);
typedef int (*fn_by_index)(unsigned int, nvml_device *);
typedef int (*fn_by_bus)(const char *, nvml_device *);
typedef int (*fn_energy)(nvml_device, unsigned long long *);

struct Nvml {
    void *h = nullptr;
    fn_by_index by_index = nullptr;
    fn_by_bus by_bus = nullptr;
    fn_energy energy = nullptr;
    bool ok = false;
};

std::mutex g_mu;
Nvml g_nvml;
bool g_tried = false;

nla_status eerr(nla_status s, const char *m) {
    nla_set_last_error(m);
    return s;
}

// Open NVML once (path: the argument, else NLA_NVML_LIB, else libnvidia-ml.so.1).
nla_status open_locked(const char *path) {
    if (g_nvml.ok) return NLA_OK;
    if (g_tried && !path) return eerr(NLA_ERR_UNSUPPORTED, "energy observer: NVML is not available");
    g_tried = true;
    const char *p = path ? path : getenv("NLA_NVML_LIB");
    void *h = dlopen(p ? p : "libnvidia-ml.so.1", RTLD_NOW | RTLD_LOCAL);
    if (!h) return eerr(NLA_ERR_UNSUPPORTED, "energy observer: cannot load NVML");
    fn_init init = reinterpret_cast<fn_init>(dlsym(h, "nvmlInit_v2"));
    Nvml n;
    n.h = h;
    n.by_index = reinterpret_cast<fn_by_index>(dlsym(h, "nvmlDeviceGetHandleByIndex_v2"));
    n.by_bus = reinterpret_cast<fn_by_bus>(dlsym(h, "nvmlDeviceGetHandleByPciBusId_v2"));
    n.energy = reinterpret_cast<fn_energy>(dlsym(h, "nvmlDeviceGetTotalEnergyConsumption"));
    if (!init || !n.by_index || !n.energy || init() != 0) {
        dlclose(h);
        return eerr(NLA_ERR_UNSUPPORTED, "energy observer: NVML lacks the energy counter");
    }
    n.ok = true;
    g_nvml = n;
    return NLA_OK;
}

nla_status read_handle(nvml_device d, unsigned long long *mj) {
    if (g_nvml.energy(d, mj) != 0) return eerr(NLA_ERR_UNSUPPORTED, "energy observer: counter not supported");
    return NLA_OK;
}

}  // namespace

extern "C" {

nla_status kt_energy_open(const char *nvml_path) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (nvml_path && g_nvml.ok) {  // an explicit library replaces the one in use
        g_nvml = Nvml();
        g_tried = false;
    }
    return open_locked(nvml_path);
}

nla_status kt_energy_read_index(unsigned int index, unsigned long long *millijoules) {
    if (!millijoules) return eerr(NLA_ERR_ARG, "null argument");
    std::lock_guard<std::mutex> lk(g_mu);
    nla_status s = open_locked(nullptr);
    if (s != NLA_OK) return s;
    nvml_device d = nullptr;
    if (g_nvml.by_index(index, &d) != 0) return eerr(NLA_ERR_ARG, "energy observer: no such NVML device");
    return read_handle(d, millijoules);
}

nla_status kt_energy_read(unsigned long long *millijoules) {
    if (!millijoules) return eerr(NLA_ERR_ARG, "null argument");
    int dev = 0;
    char bus[32] = {0};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetPCIBusId(bus, (int)sizeof bus, dev) != cudaSuccess) {
        cudaGetLastError();
        return eerr(NLA_ERR_CUDA, "energy observer: no current CUDA device");
    }
    std::lock_guard<std::mutex> lk(g_mu);
    nla_status s = open_locked(nullptr);
    if (s != NLA_OK) return s;
    nvml_device d = nullptr;
    // the current device by its PCI bus id (CUDA and NVML may number devices differently)
    if (!g_nvml.by_bus || g_nvml.by_bus(bus, &d) != 0) return eerr(NLA_ERR_UNSUPPORTED, "energy observer: device not found");
    return read_handle(d, millijoules);
}

}  // extern "C"
