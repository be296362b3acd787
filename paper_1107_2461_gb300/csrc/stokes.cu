// Semi-direct Stokes inverse (Sec. 2).
#include "fdi_internal.h"

extern "C" fdi_status fdi_stokes_solve(fdi_plan* plan, double dt, double Re, const double* const f[3],
                                       double* const u[3], double* p, fdi_stream_t stream) {
  fdi::set_error("Stokes solve not built yet");
  return FDI_ERR_UNSUPPORTED;
}
