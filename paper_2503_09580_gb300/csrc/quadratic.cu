// Quadratic operator Q(f,f) (Eq. (2.14)); implemented in a later step.
#include "lbo_internal.h"

namespace lbo {
void free_quadratic(lbo_plan* p) { (void)p; }
}  // namespace lbo

extern "C" lbo_status lbo_apply_quadratic(lbo_plan* p, const double* f, double* out, int batch) {
  (void)p; (void)f; (void)out; (void)batch;
  return LBO_EUNSUPPORTED;
}
