// Entry points whose kernels live in later translation units.
#include "internal.h"

using namespace qs;

extern "C" {

qs_status sv_grad(qs_state_t, const qs_gate*, size_t, const double*, int, int, double*, double*) {
  set_error("sv_grad not built");
  return QS_EUNSUPPORTED;
}

}  // extern "C"
