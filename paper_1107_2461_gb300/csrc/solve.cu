// Solve orchestration: the Helmholtz / Laplace inverse on one field of a plan.
//
// TPT (Sec. 3, end): forward transforms along x and y (E_x^{-1}, E_y^{-1}),
// Thomas along z per (x-mode, y-mode) line, back transforms (E_y, E_x).
// TPF (Eq. 29): forward transforms in all three directions, divide by the
// shifted eigenvalue sums (Eq. 26-28), back transforms.
//
// Both are exact inverses of the assembled operator up to rounding; the
// residual r = b - A u is evaluated with the finite-volume stencil and, while
// ||r||/||b|| exceeds the tolerance, a correction A d = r is solved by the same
// direct method and added (iterative refinement).  Every refinement kernel
// reads a device "done" flag and returns at once when the previous check has
// converged, so the whole solve is enqueued without a host round trip.
#include <cmath>

#include "fdi_internal.h"

namespace fdi {

#define FDI_TRY(expr)            \
  do {                           \
    fdi_status _s = (expr);      \
    if (_s != FDI_OK) return _s; \
  } while (0)

fdi_status validate_field_args(const fdi_plan* p, int field, double sigma, double lambda) {
  if (!p) return FDI_ERR_INVALID_ARG;
  if (field < 0 || field >= p->nfields) {
    set_error("field not present in this plan");
    return FDI_ERR_INVALID_ARG;
  }
  if (!std::isfinite(sigma) || !std::isfinite(lambda) || sigma < 0.0 || lambda < 0.0) {
    set_error("sigma and lambda must be finite and >= 0");
    return FDI_ERR_INVALID_ARG;
  }
  if (sigma == 0.0 && lambda == 0.0) {
    set_error("sigma = lambda = 0 is the zero operator");
    return FDI_ERR_INVALID_ARG;
  }
  if (sigma == 0.0 && field != FDI_FIELD_CELL) {
    set_error("the Laplace problem (sigma = 0) is defined on the cell field only");
    return FDI_ERR_INVALID_ARG;
  }
  return FDI_OK;
}

namespace {

// One direct solve in FP64: out (+)= A^{-1} in.
fdi_status solve_once_f64(fdi_plan* p, const Field& f, double sigma, double lambda, const double* in,
                          double* out, bool accumulate, const int* skip, cudaStream_t s) {
  const int nx = f.n[0], ny = f.n[1], nz = f.n[2];
  double* t0 = p->ws[0];
  double* t1 = p->ws[1];
  double* t2 = p->ws[2];
  const Axis* ax = f.ax[0];
  const Axis* ay = f.ax[1];
  const Axis* az = f.ax[2];
  FDI_TRY(launch_lines_f64(p, in, t0, ax->Einv, nx, nx, (long long)ny * nz, false, skip, s));
  FDI_TRY(launch_slab_f64(p, t0, t1, ay->Einv, ny, ny, nx, nz, skip, s));
  if (p->thomas_axis == 2) {
    FDI_TRY(launch_thomas_f64(p, f, sigma, lambda, t1, t0, t2, skip, s));
    FDI_TRY(launch_slab_f64(p, t0, t1, ay->E, ny, ny, nx, nz, skip, s));
    FDI_TRY(launch_lines_f64(p, t1, out, ax->E, nx, nx, (long long)ny * nz, accumulate, skip, s));
  } else {
    FDI_TRY(launch_slab_f64(p, t1, t0, az->Einv, nz, nz, (long long)nx * ny, 1, skip, s));
    FDI_TRY(launch_divide_f64(p, f, sigma, lambda, t0, skip, s));
    FDI_TRY(launch_slab_f64(p, t0, t1, az->E, nz, nz, (long long)nx * ny, 1, skip, s));
    FDI_TRY(launch_slab_f64(p, t1, t0, ay->E, ny, ny, nx, nz, skip, s));
    FDI_TRY(launch_lines_f64(p, t0, out, ax->E, nx, nx, (long long)ny * nz, accumulate, skip, s));
  }
  return FDI_OK;
}

}  // namespace

fdi_status field_solve(fdi_plan* p, int field, double sigma, double lambda, const double* rhs, double* out,
                       cudaStream_t s) {
  FDI_TRY(validate_field_args(p, field, sigma, lambda));
  if (!rhs || !out) return FDI_ERR_INVALID_ARG;
  if (p->prec != FDI_PREC_FP64) return mixed_field_solve(p, field, sigma, lambda, rhs, out, s);
  const Field& f = p->fields[field];
  FDI_TRY(launch_reset_status(p, s));
  const double* b = rhs;
  if (out == rhs) {
    FDI_CUDA_TRY(cudaMemcpyAsync(p->ws[4], rhs, f.P * sizeof(double), cudaMemcpyDeviceToDevice, s));
    b = p->ws[4];
  }
  const bool singular = sigma == 0.0 && f.zero_flux_all;
  if (singular) FDI_TRY(launch_mean_f64(p, f, b, s));
  const int* done = &p->d_status->done;
  double* r = p->ws[3];
  FDI_TRY(solve_once_f64(p, f, sigma, lambda, b, out, false, nullptr, s));
  FDI_TRY(launch_residual_f64(p, f, sigma, lambda, b, out, r, singular, nullptr, s));
  FDI_TRY(launch_finish_residual(p, 0, true, 0, nullptr, s));
  for (int k = 0; k < p->max_refine; ++k) {
    FDI_TRY(solve_once_f64(p, f, sigma, lambda, r, out, true, done, s));
    FDI_TRY(launch_residual_f64(p, f, sigma, lambda, b, out, r, singular, done, s));
    FDI_TRY(launch_finish_residual(p, 0, false, 1, done, s));
  }
  return FDI_OK;
}

void invalidate_graph(fdi_plan* p) {
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  p->gexec = nullptr;
  p->gkey_valid = false;
  p->glaunches = 0;
  if (p->kgraph) cudaGraphExecDestroy(p->kgraph);
  p->kgraph = nullptr;
  p->kgraph_precond = -1;
}

namespace {

bool same_key(const fdi_plan::GraphKey& a, const fdi_plan::GraphKey& b) {
  return a.field == b.field && a.sigma == b.sigma && a.lambda == b.lambda && a.rhs == b.rhs && a.out == b.out &&
         a.s == b.s;
}

// Field solve through the graph cache: the first call with new arguments runs
// eagerly, the second identical call is captured (stream capture of the same
// launch sequence) and every later identical call is one graph launch.  The
// legacy default stream cannot be captured and timed plans need their events,
// so both run eagerly.
fdi_status field_solve_entry(fdi_plan* p, int field, double sigma, double lambda, const double* rhs, double* out,
                             cudaStream_t s) {
  if (!p) return FDI_ERR_INVALID_ARG;
  p->launches = 0;
  if (!p->use_graphs || p->timing || s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread)
    return field_solve(p, field, sigma, lambda, rhs, out, s);
  fdi_plan::GraphKey key;
  key.field = field;
  key.sigma = sigma;
  key.lambda = lambda;
  key.rhs = rhs;
  key.out = out;
  key.s = s;
  if (p->gkey_valid && same_key(key, p->gkey) && p->gexec) {
    FDI_CUDA_TRY(cudaGraphLaunch(p->gexec, s));
    p->launches = p->glaunches;
    return FDI_OK;
  }
  if (!p->gkey_valid || !same_key(key, p->gkey)) {
    invalidate_graph(p);
    fdi_status st = field_solve(p, field, sigma, lambda, rhs, out, s);
    if (st == FDI_OK) {
      p->gkey = key;
      p->gkey_valid = true;
    }
    return st;
  }
  // second call with these arguments: capture, instantiate, launch
  FDI_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  fdi_status st = field_solve(p, field, sigma, lambda, rhs, out, s);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (st != FDI_OK || e != cudaSuccess || g == nullptr) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    invalidate_graph(p);
    if (st != FDI_OK) return st;
    return field_solve(p, field, sigma, lambda, rhs, out, s);  // capture refused: eager
  }
  const long long n_launch = p->launches;
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    invalidate_graph(p);
    return field_solve(p, field, sigma, lambda, rhs, out, s);
  }
  p->gexec = ex;
  p->glaunches = n_launch;
  FDI_CUDA_TRY(cudaGraphLaunch(p->gexec, s));
  p->launches = n_launch;
  return FDI_OK;
}

}  // namespace

}  // namespace fdi

using namespace fdi;

extern "C" {

fdi_status fdi_field_solve(fdi_plan* plan, fdi_field field, double sigma, double lambda, const double* rhs,
                           double* out, fdi_stream_t stream) {
  fdi_status st = validate_field_args(plan, (int)field, sigma, lambda);
  if (st != FDI_OK) return st;
  return field_solve_entry(plan, (int)field, sigma, lambda, rhs, out, (cudaStream_t)stream);
}

fdi_status fdi_helmholtz_solve(fdi_plan* plan, double lambda, const double* rhs, double* out,
                               fdi_stream_t stream) {
  fdi_status st = validate_field_args(plan, FDI_FIELD_CELL, 1.0, lambda);
  if (st != FDI_OK) return st;
  return field_solve_entry(plan, FDI_FIELD_CELL, 1.0, lambda, rhs, out, (cudaStream_t)stream);
}

fdi_status fdi_laplace_solve(fdi_plan* plan, const double* rhs, double* out, fdi_stream_t stream) {
  fdi_status st = validate_field_args(plan, FDI_FIELD_CELL, 0.0, 1.0);
  if (st != FDI_OK) return st;
  return field_solve_entry(plan, FDI_FIELD_CELL, 0.0, 1.0, rhs, out, (cudaStream_t)stream);
}

fdi_status fdi_helmholtz_solve_batched(fdi_plan* const* plans, const double* lambdas, const double* const* rhs,
                                       double* const* out, int count, fdi_stream_t stream) {
  if (count < 0 || (count > 0 && (!plans || !lambdas || !rhs || !out))) return FDI_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i) {
    fdi_status st = validate_field_args(plans[i], FDI_FIELD_CELL, 1.0, lambdas[i]);
    if (st != FDI_OK) return st;
    if (!rhs[i] || !out[i]) return FDI_ERR_INVALID_ARG;
  }
  for (int i = 0; i < count; ++i) {
    fdi_status st = field_solve_entry(plans[i], FDI_FIELD_CELL, 1.0, lambdas[i], rhs[i], out[i],
                                      (cudaStream_t)stream);
    if (st != FDI_OK) return st;
  }
  return FDI_OK;
}

fdi_status fdi_plan_set_graphs(fdi_plan* plan, int on) {
  if (!plan) return FDI_ERR_INVALID_ARG;
  plan->use_graphs = on != 0;
  invalidate_graph(plan);
  return FDI_OK;
}

}  // extern "C"
