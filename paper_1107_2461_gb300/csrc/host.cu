// Field solves whose right-hand sides and solutions live in host memory.
//
// A sequence of independent solves (Sec. 3 direct inverse with refinement, one
// per right-hand side) is pipelined over three streams: while solve s runs on
// the compute stream, the host-to-device copy of right-hand side s+1 runs on
// one copy stream and the device-to-host copy of solution s-1 on the other.
// Two device staging buffers per direction alternate between consecutive
// solves; events order each buffer's reuse (a right-hand side buffer is
// refilled once the solve two steps back has finished with it, a solution
// buffer is rewritten once its copy to the host has finished).  The solve
// itself is the graph-cached field solve, so the two alternating argument
// sets each replay one captured graph.  Each solve's device status record is
// copied into a per-solve array, so every solve's outcome is reported.
#include <algorithm>
#include <string>

#include "fdi_internal.h"

namespace fdi {

#define FDI_TRY(expr)            \
  do {                           \
    fdi_status _s = (expr);      \
    if (_s != FDI_OK) return _s; \
  } while (0)

void free_host_staging(fdi_plan* p) {
  for (double*& b : p->hstage) {
    if (b) cudaFree(b);
    b = nullptr;
  }
  p->hstage_len = 0;
  for (cudaStream_t& st : p->hcopy) {
    if (st) cudaStreamDestroy(st);
    st = nullptr;
  }
  for (cudaEvent_t& e : p->hev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
  if (p->d_hstat) cudaFree(p->d_hstat);
  if (p->h_hstat) cudaFreeHost(p->h_hstat);
  p->d_hstat = nullptr;
  p->h_hstat = nullptr;
  p->hstat_cap = 0;
}

namespace {

// staging buffers of P doubles, streams, events and a status array for
// `count` solves (allocated on first use, grown when needed)
fdi_status ensure_host_staging(fdi_plan* p, long long P, int count) {
  if (p->hstage_len < P) {
    for (double*& b : p->hstage) {
      if (b) cudaFree(b);
      b = nullptr;
    }
    p->hstage_len = 0;
    for (double*& b : p->hstage) FDI_CUDA_TRY(cudaMalloc(&b, (size_t)P * sizeof(double)));
    p->hstage_len = P;
  }
  for (cudaStream_t& st : p->hcopy)
    if (!st) FDI_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  for (cudaEvent_t& e : p->hev)
    if (!e) FDI_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  if (p->hstat_cap < count) {
    if (p->d_hstat) cudaFree(p->d_hstat);
    if (p->h_hstat) cudaFreeHost(p->h_hstat);
    p->d_hstat = nullptr;
    p->h_hstat = nullptr;
    p->hstat_cap = 0;
    const int cap = std::max(count, 64);
    FDI_CUDA_TRY(cudaMalloc(&p->d_hstat, (size_t)cap * sizeof(DevStatus)));
    FDI_CUDA_TRY(cudaMallocHost(&p->h_hstat, (size_t)cap * sizeof(DevStatus)));
    p->hstat_cap = cap;
  }
  return FDI_OK;
}

fdi_status enqueue_pipeline(fdi_plan* p, int field, double sigma, double lambda, const double* const* h_rhs,
                            double* const* h_out, int count, cudaStream_t s) {
  const long long P = p->fields[field].P;
  const size_t bytes = (size_t)P * sizeof(double);
  cudaStream_t h2d = p->hcopy[0], d2h = p->hcopy[1];
  cudaEvent_t* ev_in = p->hev + 0;
  cudaEvent_t* ev_solved = p->hev + 2;
  cudaEvent_t* ev_out = p->hev + 4;
  cudaEvent_t ev_start = p->hev[6];
  // the copy streams start after the work already queued on the compute stream
  FDI_CUDA_TRY(cudaEventRecord(ev_start, s));
  FDI_CUDA_TRY(cudaStreamWaitEvent(h2d, ev_start, 0));
  FDI_CUDA_TRY(cudaStreamWaitEvent(d2h, ev_start, 0));
  for (int i = 0; i < count; ++i) {
    const int b = i & 1;
    double* d_in = p->hstage[b];
    double* d_out = p->hstage[2 + b];
    // right-hand side i into buffer b, once solve i-2 no longer reads it
    if (i >= 2) FDI_CUDA_TRY(cudaStreamWaitEvent(h2d, ev_solved[b], 0));
    FDI_CUDA_TRY(cudaMemcpyAsync(d_in, h_rhs[i], bytes, cudaMemcpyHostToDevice, h2d));
    FDI_CUDA_TRY(cudaEventRecord(ev_in[b], h2d));
    // solve i, once its input has arrived and solution i-2 has left buffer b
    FDI_CUDA_TRY(cudaStreamWaitEvent(s, ev_in[b], 0));
    if (i >= 2) FDI_CUDA_TRY(cudaStreamWaitEvent(s, ev_out[b], 0));
    FDI_TRY(field_solve_entry(p, field, sigma, lambda, d_in, d_out, s));
    FDI_CUDA_TRY(cudaMemcpyAsync(p->d_hstat + i, p->d_status, sizeof(DevStatus), cudaMemcpyDeviceToDevice, s));
    FDI_CUDA_TRY(cudaEventRecord(ev_solved[b], s));
    // solution i back to the host
    FDI_CUDA_TRY(cudaStreamWaitEvent(d2h, ev_solved[b], 0));
    FDI_CUDA_TRY(cudaMemcpyAsync(h_out[i], d_out, bytes, cudaMemcpyDeviceToHost, d2h));
    FDI_CUDA_TRY(cudaEventRecord(ev_out[b], d2h));
  }
  // the compute stream ends after the last copy to the host
  FDI_CUDA_TRY(cudaEventRecord(ev_start, d2h));
  FDI_CUDA_TRY(cudaStreamWaitEvent(s, ev_start, 0));
  FDI_CUDA_TRY(cudaMemcpyAsync(p->h_hstat, p->d_hstat, (size_t)count * sizeof(DevStatus), cudaMemcpyDeviceToHost,
                               s));
  return FDI_OK;
}

}  // namespace
}  // namespace fdi

extern "C" fdi_status fdi_field_solve_host(fdi_plan* plan, fdi_field field, double sigma, double lambda,
                                           const double* const* h_rhs, double* const* h_out, int count,
                                           double* rel_residual, fdi_stream_t stream) {
  using namespace fdi;
  fdi_status st = validate_field_args(plan, (int)field, sigma, lambda);
  if (st != FDI_OK) return st;
  if (count < 0 || (count > 0 && (!h_rhs || !h_out))) return FDI_ERR_INVALID_ARG;
  for (int i = 0; i < count; ++i)
    if (!h_rhs[i] || !h_out[i]) {
      set_error("fdi_field_solve_host: null host array");
      return FDI_ERR_INVALID_ARG;
    }
  if (count == 0) return FDI_OK;
  FDI_TRY(ensure_host_staging(plan, plan->fields[(int)field].P, count));
  // the legacy default stream would serialise with the copy streams' work in
  // ways the events already order; the plan's own compute stream replaces it
  cudaStream_t s = (cudaStream_t)stream;
  if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread) {
    FDI_CUDA_TRY(cudaStreamSynchronize(s));
    s = plan->hcopy[2];
  }
  st = enqueue_pipeline(plan, (int)field, sigma, lambda, h_rhs, h_out, count, s);
  // blocking: every copy queued above finishes before the host arrays are
  // handed back (also after an enqueue error, so no copy outlives the call)
  const cudaError_t e = cudaStreamSynchronize(s);
  cudaStreamSynchronize(plan->hcopy[0]);
  cudaStreamSynchronize(plan->hcopy[1]);
  if (st != FDI_OK) return st;
  if (e != cudaSuccess) {
    set_error(std::string("fdi_field_solve_host: ") + cudaGetErrorString(e));
    return FDI_ERR_CUDA;
  }
  int kerr = 0;
  if (plan->d_err) FDI_CUDA_TRY(cudaMemcpy(&kerr, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  fdi_status first_bad = FDI_OK;
  std::string bad_msg;
  for (int i = 0; i < count; ++i) {
    const DevStatus& ds = plan->h_hstat[i];
    if (rel_residual) rel_residual[i] = ds.rel_res;
    const fdi_status si = solve_status(plan, ds, kerr);
    if (si != FDI_OK && first_bad == FDI_OK) {
      first_bad = si;
      bad_msg = "right-hand side " + std::to_string(i) + ": " + fdi_last_error_message();
    }
  }
  if (first_bad != FDI_OK) set_error(bad_msg);
  return first_bad;
}
