// Tensor-core (tcgen05) paths.  Placeholder until the tcgen05 kernels land.
#include "internal.h"

namespace hm {
hess_status run_opg_tc(hess_mlp*, const void*, const void*, int64_t, bool, void*) {
  return set_error(HESS_ERR_UNSUPPORTED, "tensor-core OPG not built");
}
hess_status run_hessian_tc(hess_mlp*, const void*, const void*, int64_t, bool, void*) {
  return set_error(HESS_ERR_UNSUPPORTED, "tensor-core Hessian not built");
}
}  // namespace hm
