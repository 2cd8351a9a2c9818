// Ridge least-squares fit of Eq. 63a (design matrix, normal equations, Cholesky).
#include <cuda_runtime.h>

#include "pod_internal.h"

extern "C" int pod_fit(pod_handle* h, const pod_system* batch, const double* E_ref, const double* F_ref,
                       const pod_fit_opts* opts, double* c_out, double* mae_E, double* mae_F) {
  if (!h) return POD_EINVAL;
  (void)batch; (void)E_ref; (void)F_ref; (void)opts; (void)c_out; (void)mae_E; (void)mae_F;
  return h->fail(POD_EINVAL, "pod_fit: not built yet");
}
