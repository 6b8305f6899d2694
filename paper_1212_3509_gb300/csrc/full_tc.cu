// Full format on tcgen05 tensor cores (split-precision TF32x3 / BF16x3).
#include "internal.h"

namespace demag {

demag_status tc_prepare(demag_plan* P, demag_precision prec, cudaStream_t st) {
  (void)prec; (void)st;
  return set_error(P, DEMAG_EUNSUPPORTED, "tensor-core forms are not built yet");
}
demag_status tc_forward(demag_plan* P, const float*, float*, demag_precision prec, cudaStream_t st) {
  return tc_prepare(P, prec, st);
}
demag_status tc_adjoint(demag_plan* P, const float*, float*, demag_precision prec, cudaStream_t st) {
  return tc_prepare(P, prec, st);
}
size_t tc_workspace_bytes(const demag_plan*, demag_precision) { return 0; }
void tc_destroy(demag_plan*) {}

}  // namespace demag
