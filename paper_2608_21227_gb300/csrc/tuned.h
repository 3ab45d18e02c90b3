// tuned.h -- internal hook between the C ABI and the tuner's installed table.
#pragma once

#include "../../include/nla.h"

#ifdef __cplusplus
extern "C" {
#endif

// Look up the installed best configuration for a problem (side 0 = QR-side
// update, 1 = LQ-side update).  Returns 1 and fills *out when the table (see
// kt_load_config) has an entry for this dtype/update, else 0.
int nla_tuned_lookup(int m, int n, int dtype, int update, int side, nla_cfg *out);

// Record the message returned by nla_last_error() on this thread.
void nla_set_last_error(const char *msg);

#ifdef __cplusplus
}
#endif
