// batched.cu -- many small matrices of uneven shapes in one persistent launch.
#include "../../include/nla.h"
#include "common.cuh"
#include "kernels.cuh"

extern "C" {

nla_status nla_gesvd_vals_batched_workspace(int batch, nla_dtype dtype, const int *hM, const int *hN,
                                            size_t *bytes) {
    (void)batch;
    (void)dtype;
    (void)hM;
    (void)hN;
    if (bytes) *bytes = 0;
    return NLA_ERR_UNSUPPORTED;
}

nla_status nla_gesvd_vals_batched(int batch, nla_dtype dtype, const int *hM, const int *hN, const int *hLda,
                                  void *const *dA_array, void *const *dS_array, void *dWork, size_t work_bytes,
                                  int *dInfo, const nla_opts *opts, nla_stream_t stream) {
    (void)batch; (void)dtype; (void)hM; (void)hN; (void)hLda; (void)dA_array; (void)dS_array;
    (void)dWork; (void)work_bytes; (void)dInfo; (void)opts; (void)stream;
    return NLA_ERR_UNSUPPORTED;
}

}  // extern "C"
