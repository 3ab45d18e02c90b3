// update_tc.cu -- mixed-precision trailing update (TF32 / BF16 operands on the
// tensor cores, FP32 accumulation, FP64 matrix).
#include "common.cuh"
#include "kernels.cuh"

namespace nla {

bool trail_tc_available() { return false; }

size_t trail_tc_scratch_bytes(int M, int N, int nb) {
    (void)M;
    (void)N;
    (void)nb;
    return 256;
}

cudaError_t trail_left_tc(double *, long, int, int, const double *, long, int, const double *, int, void *,
                          size_t, cudaStream_t) {
    return cudaErrorNotSupported;
}

cudaError_t trail_right_tc(double *, long, int, int, const double *, long, int, const double *, int, void *,
                           size_t, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace nla
