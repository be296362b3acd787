// Mixed-precision path (split tensor-core transforms + double-float refinement).
#include "fdi_internal.h"

namespace fdi {

fdi_status mixed_setup(fdi_plan* p) { return FDI_OK; }

fdi_status mixed_field_solve(fdi_plan* p, int field, double sigma, double lambda, const double* rhs,
                             double* out, cudaStream_t s) {
  set_error("mixed precision path not built yet");
  return FDI_ERR_UNSUPPORTED;
}

}  // namespace fdi
