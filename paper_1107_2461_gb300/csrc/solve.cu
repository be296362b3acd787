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
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "fdi_internal.h"
#include "resident.h"

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
  if (sigma == 0.0 && p->cyl && p->fields[0].zero_flux_all) {
    set_error("the zero-flux Laplacian of a cylindrical plan is singular; not handled");
    return FDI_ERR_UNSUPPORTED;
  }
  return FDI_OK;
}

namespace {

// One direct solve in FP64: out (+)= A^{-1} in.
fdi_status solve_once_f64(fdi_plan* p, int field, double sigma, double lambda, const double* in, double* out,
                          bool accumulate, const int* skip, cudaStream_t s) {
  const Field& f = p->fields[field];
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
    FDI_TRY(launch_thomas_f64(p, f, sigma, lambda, field, t1, t0, t2, skip, s));
    FDI_TRY(launch_slab_f64(p, t0, t1, ay->E, ny, ny, nx, nz, skip, s));
    FDI_TRY(launch_lines_f64(p, t1, out, ax->E, nx, nx, (long long)ny * nz, accumulate, skip, s));
  } else if (p->cyl) {
    // cylindrical TPF (Eq. 45-46): the radial transform of theta mode j uses
    // that mode's own eigenbasis, the divide its own eigenvalues
    FDI_TRY(launch_modes_f64(p, t1, t0, p->cyl_Eri, nz, nx, ny, skip, s));
    FDI_TRY(launch_divide_modes_f64(p, f, sigma, lambda, t0, skip, s));
    FDI_TRY(launch_modes_f64(p, t0, t1, p->cyl_Er, nz, nx, ny, skip, s));
    FDI_TRY(launch_slab_f64(p, t1, t0, ay->E, ny, ny, nx, nz, skip, s));
    FDI_TRY(launch_lines_f64(p, t0, out, ax->E, nx, nx, (long long)ny * nz, accumulate, skip, s));
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

namespace {

fdi_status field_solve_internal(fdi_plan* p, int field, double sigma, double lambda, const double* rhs, double* out,
                                cudaStream_t s) {
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
  FDI_TRY(solve_once_f64(p, field, sigma, lambda, b, out, false, nullptr, s));
  FDI_TRY(launch_residual_f64(p, f, sigma, lambda, b, out, r, singular, nullptr, s));
  FDI_TRY(launch_finish_residual(p, 0, true, 0, nullptr, s));
  for (int k = 0; k < p->max_refine; ++k) {
    FDI_TRY(solve_once_f64(p, field, sigma, lambda, r, out, true, done, s));
    FDI_TRY(launch_residual_f64(p, f, sigma, lambda, b, out, r, singular, done, s));
    FDI_TRY(launch_finish_residual(p, 0, false, 1, done, s));
  }
  return FDI_OK;
}

}  // namespace

fdi_status field_solve(fdi_plan* p, int field, double sigma, double lambda, const double* rhs, double* out,
                       cudaStream_t s) {
  FDI_TRY(validate_field_args(p, field, sigma, lambda));
  if (!rhs || !out) return FDI_ERR_INVALID_ARG;
  if (p->tstage[0] == nullptr) return field_solve_internal(p, field, sigma, lambda, rhs, out, s);
  // Thomas along x or y: solve on the copy with that axis outermost
  FDI_TRY(launch_axis_permute(p, rhs, p->tstage[0], true, s));
  FDI_TRY(field_solve_internal(p, field, sigma, lambda, p->tstage[0], p->tstage[1], s));
  return launch_axis_permute(p, p->tstage[1], out, false, s);
}

// Autotuned Thomas configurations per (grid shape, precision),
// applied to plans created later with the same shape.
namespace {
struct TuneKey {
  int n0, n1, n2, prec, grid;
  bool operator<(const TuneKey& o) const {
    return std::tie(n0, n1, n2, prec, grid) < std::tie(o.n0, o.n1, o.n2, o.prec, o.grid);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
TuneKey tune_key(const fdi_plan* p) { return TuneKey{p->n[0], p->n[1], p->n[2], (int)p->prec, (int)p->grid}; }
}  // namespace

void forget_batch_graph(const fdi_plan* p);

void remember_tuning(const fdi_plan* p) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[tune_key(p)] = p->thomas_tl;
}

void apply_tuning(fdi_plan* p) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(tune_key(p));
  if (it != g_tune.end()) p->thomas_tl = it->second;
}

void invalidate_graph(fdi_plan* p) {
  for (fdi_plan::GraphSlot& g : p->gslots) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g = fdi_plan::GraphSlot{};
  }
  if (p->kgraph) cudaGraphExecDestroy(p->kgraph);
  p->kgraph = nullptr;
  p->kgraph_precond = -1;
  forget_batch_graph(p);
}

namespace {

bool same_key(const fdi_plan::GraphKey& a, const fdi_plan::GraphKey& b) {
  return a.field == b.field && a.sigma == b.sigma && a.lambda == b.lambda && a.rhs == b.rhs && a.out == b.out &&
         a.s == b.s;
}

}  // namespace

// Field solve through the graph cache: the first call with new arguments runs
// eagerly, the second identical call is captured (stream capture of the same
// launch sequence) and every later identical call is one graph launch.  The
// cache keeps the graphs of the last few distinct argument sets.  The legacy
// default stream cannot be captured and timed plans need their events, so both
// run eagerly.
fdi_status field_solve_entry(fdi_plan* p, int field, double sigma, double lambda, const double* rhs, double* out,
                             cudaStream_t s) {
  if (!p) return FDI_ERR_INVALID_ARG;
  p->launches = 0;
  p->kloop_body_launches = 0;
  if (!p->use_graphs || p->timing || s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread)
    return field_solve(p, field, sigma, lambda, rhs, out, s);
  fdi_plan::GraphKey key;
  key.field = field;
  key.sigma = sigma;
  key.lambda = lambda;
  key.rhs = rhs;
  key.out = out;
  key.s = s;
  fdi_plan::GraphSlot* g = nullptr;
  for (fdi_plan::GraphSlot& c : p->gslots)
    if (c.valid && same_key(key, c.key)) g = &c;
  if (g && g->exec) {
    g->last_use = ++p->gclock;
    FDI_CUDA_TRY(cudaGraphLaunch(g->exec, s));
    p->launches = g->launches;
    return FDI_OK;
  }
  if (!g) {
    // first call with these arguments: eager; remember the key in a free or
    // the least recently used slot
    g = &p->gslots[0];
    for (fdi_plan::GraphSlot& c : p->gslots) {
      if (!c.valid) {
        g = &c;
        break;
      }
      if (c.last_use < g->last_use) g = &c;
    }
    if (g->exec) cudaGraphExecDestroy(g->exec);
    *g = fdi_plan::GraphSlot{};
    fdi_status st = field_solve(p, field, sigma, lambda, rhs, out, s);
    if (st == FDI_OK) {
      g->key = key;
      g->valid = true;
      g->last_use = ++p->gclock;
    }
    return st;
  }
  // second call with these arguments: capture, instantiate, launch
  g->last_use = ++p->gclock;
  FDI_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  fdi_status st = field_solve(p, field, sigma, lambda, rhs, out, s);
  cudaGraph_t gr = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &gr);
  if (st != FDI_OK || e != cudaSuccess || gr == nullptr) {
    if (gr) cudaGraphDestroy(gr);
    cudaGetLastError();
    *g = fdi_plan::GraphSlot{};
    if (st != FDI_OK) return st;
    return field_solve(p, field, sigma, lambda, rhs, out, s);  // capture refused: eager
  }
  const long long n_launch = p->launches;
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, gr, 0);
  cudaGraphDestroy(gr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *g = fdi_plan::GraphSlot{};
    return field_solve(p, field, sigma, lambda, rhs, out, s);
  }
  g->exec = ex;
  g->launches = n_launch;
  FDI_CUDA_TRY(cudaGraphLaunch(g->exec, s));
  p->launches = n_launch;
  return FDI_OK;
}

namespace {

// ---- batched solves: independent plans run concurrently on a pool of streams ----

constexpr int kBatchStreams = 32;

struct StreamPool {
  cudaStream_t st[kBatchStreams] = {};
  cudaEvent_t done[kBatchStreams] = {};
  cudaEvent_t fork = nullptr;
  bool ok = false;
};

std::mutex g_pool_mu;
std::map<int, StreamPool> g_pools;

StreamPool* stream_pool() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  StreamPool& sp = g_pools[dev];
  if (!sp.ok) {
    for (int k = 0; k < kBatchStreams; ++k) {
      if (cudaStreamCreateWithFlags(&sp.st[k], cudaStreamNonBlocking) != cudaSuccess) return nullptr;
      if (cudaEventCreateWithFlags(&sp.done[k], cudaEventDisableTiming) != cudaSuccess) return nullptr;
    }
    if (cudaEventCreateWithFlags(&sp.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    sp.ok = true;
  }
  return &sp;
}

// Fork from s onto the pool, one stream per distinct plan (a plan appearing
// twice keeps one stream, so its workspace is used in order), join back on s.
fdi_status enqueue_batch(StreamPool* sp, fdi_plan* const* plans, const double* lambdas, const double* const* rhs,
                         double* const* out, int count, cudaStream_t s) {
  FDI_CUDA_TRY(cudaEventRecord(sp->fork, s));
  std::vector<int> lane(count, -1);
  bool used[kBatchStreams] = {false};
  // small grids: resident launches of up to kResMaxJobs solves on pool stream
  // 0 (a plan repeated in the batch goes to a later launch, in order); the
  // other plans one stream each on streams 1...
  std::vector<char> res(count, 0);
  for (int i = 0; i < count; ++i)
    res[i] = (plans[i]->tstage[0] == nullptr && resident_eligible(plans[i], FDI_FIELD_CELL) &&
              validate_field_args(plans[i], FDI_FIELD_CELL, 1.0, lambdas[i]) == FDI_OK) ? 1 : 0;
  {
    std::vector<char> taken(count, 0);
    for (;;) {
      std::vector<ResJob> jobs;
      std::vector<fdi_plan*> in_launch;
      for (int i = 0; i < count && (int)jobs.size() < kResMaxJobs; ++i) {
        if (!res[i] || taken[i]) continue;
        bool dup = false;
        for (fdi_plan* q : in_launch) dup = dup || q == plans[i];
        for (int j = 0; j < i && !dup; ++j) dup = res[j] && !taken[j] && plans[j] == plans[i];
        if (dup) continue;
        ResJob job;
        FDI_TRY(resident_describe(plans[i], FDI_FIELD_CELL, 1.0, lambdas[i], rhs[i], out[i], &job));
        jobs.push_back(job);
        in_launch.push_back(plans[i]);
        taken[i] = 1;
        plans[i]->launches = 0;
      }
      if (jobs.empty()) break;
      if (!used[0]) {
        FDI_CUDA_TRY(cudaStreamWaitEvent(sp->st[0], sp->fork, 0));
        used[0] = true;
      }
      FDI_TRY(resident_launch(in_launch[0], jobs.data(), (int)jobs.size(), sp->st[0]));
    }
  }
  int next = 0;
  for (int i = 0; i < count; ++i) {
    if (res[i]) continue;
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) {
        lane[i] = lane[j];
        break;
      }
    if (lane[i] < 0) lane[i] = 1 + (next++) % (kBatchStreams - 1);
    const int k = lane[i];
    if (!used[k]) {
      FDI_CUDA_TRY(cudaStreamWaitEvent(sp->st[k], sp->fork, 0));
      used[k] = true;
    }
    plans[i]->launches = 0;
    FDI_TRY(field_solve(plans[i], FDI_FIELD_CELL, 1.0, lambdas[i], rhs[i], out[i], sp->st[k]));
  }
  for (int k = 0; k < kBatchStreams; ++k)
    if (used[k]) {
      FDI_CUDA_TRY(cudaEventRecord(sp->done[k], sp->st[k]));
      FDI_CUDA_TRY(cudaStreamWaitEvent(s, sp->done[k], 0));
    }
  return FDI_OK;
}

// Graph of a whole batch: captured on the second call with identical
// arguments, then replayed as one launch.
struct BatchGraph {
  std::vector<fdi_plan*> plans;
  std::vector<double> lambdas;
  std::vector<const double*> rhs;
  std::vector<double*> out;
  cudaStream_t s = nullptr;
  bool seen = false;
  cudaGraphExec_t exec = nullptr;
  std::vector<long long> launches;
};

std::mutex g_batch_mu;
BatchGraph g_batch;

bool same_batch(const BatchGraph& g, fdi_plan* const* plans, const double* lambdas, const double* const* rhs,
                double* const* out, int count, cudaStream_t s) {
  if ((int)g.plans.size() != count || g.s != s) return false;
  for (int i = 0; i < count; ++i)
    if (g.plans[i] != plans[i] || g.lambdas[i] != lambdas[i] || g.rhs[i] != rhs[i] || g.out[i] != out[i]) return false;
  return true;
}

}  // namespace

// drop the batch graph if it involves this plan (plan destroyed or changed)
void forget_batch_graph(const fdi_plan* p) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (fdi_plan* q : g_batch.plans)
    if (q == p) {
      if (g_batch.exec) cudaGraphExecDestroy(g_batch.exec);
      g_batch = BatchGraph();
      return;
    }
}

fdi_status batch_solve(fdi_plan* const* plans, const double* lambdas, const double* const* rhs, double* const* out,
                       int count, cudaStream_t s) {
  StreamPool* sp = stream_pool();
  if (!sp) {
    set_error("could not create the batch stream pool");
    return FDI_ERR_CUDA;
  }
  bool graphs = s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
  for (int i = 0; i < count; ++i) graphs = graphs && plans[i]->use_graphs && !plans[i]->timing;
  std::lock_guard<std::mutex> lk(g_batch_mu);
  if (!graphs) return enqueue_batch(sp, plans, lambdas, rhs, out, count, s);
  if (same_batch(g_batch, plans, lambdas, rhs, out, count, s)) {
    if (g_batch.exec) {
      FDI_CUDA_TRY(cudaGraphLaunch(g_batch.exec, s));
      for (int i = 0; i < count; ++i) plans[i]->launches = g_batch.launches[i];
      return FDI_OK;
    }
    // second identical call: capture the fork / solves / join
    FDI_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    fdi_status st = enqueue_batch(sp, plans, lambdas, rhs, out, count, s);
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &gr);
    if (st != FDI_OK || e != cudaSuccess || !gr) {
      if (gr) cudaGraphDestroy(gr);
      cudaGetLastError();
      g_batch = BatchGraph();
      if (st != FDI_OK) return st;
      return enqueue_batch(sp, plans, lambdas, rhs, out, count, s);
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      cudaGetLastError();
      g_batch = BatchGraph();
      return enqueue_batch(sp, plans, lambdas, rhs, out, count, s);
    }
    g_batch.exec = ex;
    g_batch.launches.assign(count, 0);
    for (int i = 0; i < count; ++i) g_batch.launches[i] = plans[i]->launches;
    FDI_CUDA_TRY(cudaGraphLaunch(ex, s));
    return FDI_OK;
  }
  // new arguments: run eagerly and remember them
  if (g_batch.exec) cudaGraphExecDestroy(g_batch.exec);
  g_batch = BatchGraph();
  fdi_status st = enqueue_batch(sp, plans, lambdas, rhs, out, count, s);
  if (st == FDI_OK) {
    g_batch.plans.assign(plans, plans + count);
    g_batch.lambdas.assign(lambdas, lambdas + count);
    g_batch.rhs.assign(rhs, rhs + count);
    g_batch.out.assign(out, out + count);
    g_batch.s = s;
    g_batch.seen = true;
  }
  return st;
}

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
  if (count == 0) return FDI_OK;
  return batch_solve(plans, lambdas, rhs, out, count, (cudaStream_t)stream);
}

fdi_status fdi_plan_set_thomas_config(fdi_plan* plan, int lines_per_cta) {
  if (!plan || (lines_per_cta != 2 && lines_per_cta != 3 && lines_per_cta != 4 && lines_per_cta != 64 &&
                lines_per_cta != 128))
    return FDI_ERR_INVALID_ARG;
  if (lines_per_cta == 4 && plan->prec != FDI_PREC_FP64) {
    // FP64 recurrence with cached line factors: a cache in every workspace
    long long q = 0;
    for (int fi = 0; fi < plan->nfields; ++fi) q = std::max(q, plan->fields[fi].P);
    FDI_TRY(alloc_thomas_cache(plan, q));
    for (int c = 0; c < plan->nextra; ++c) {
      SlotSwap guard(plan, &plan->extra[c]);
      FDI_TRY(alloc_thomas_cache(plan, q));
    }
  }
  plan->thomas_tl = lines_per_cta;
  invalidate_graph(plan);
  return FDI_OK;
}

fdi_status fdi_plan_autotune(fdi_plan* plan, double lambda, const double* rhs, double* out, int reps,
                             int* thomas_tl_out, fdi_stream_t stream) {
  fdi_status st = validate_field_args(plan, FDI_FIELD_CELL, 1.0, lambda);
  if (st != FDI_OK) return st;
  if (!rhs || !out || rhs == out || reps < 1 || reps > 1000) return FDI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (plan->prec != FDI_PREC_FP64) {
    const int tls[4] = {2, 3, 64, 128};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    FDI_CUDA_TRY(cudaEventCreate(&e0));
    FDI_CUDA_TRY(cudaEventCreate(&e1));
    float best = 0.f;
    int best_t = plan->thomas_tl;
    const bool timing = plan->timing;
    plan->timing = false;
    {
      for (int ti = 0; ti < 4 && st == FDI_OK; ++ti) {
        plan->thomas_tl = tls[ti];
        st = field_solve(plan, FDI_FIELD_CELL, 1.0, lambda, rhs, out, s);  // warm-up
        if (st != FDI_OK) break;
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && st == FDI_OK; ++r) st = field_solve(plan, FDI_FIELD_CELL, 1.0, lambda, rhs, out, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          set_error("autotune: timing event failed");
          st = FDI_ERR_CUDA;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best == 0.f || ms < best) {
          best = ms;
          best_t = tls[ti];
        }
      }
    }
    plan->timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    plan->thomas_tl = best_t;
    invalidate_graph(plan);
    if (st != FDI_OK) return st;
    remember_tuning(plan);
  }
  if (thomas_tl_out) *thomas_tl_out = plan->thomas_tl;
  return FDI_OK;
}

fdi_status fdi_plan_set_graphs(fdi_plan* plan, int on) {
  if (!plan) return FDI_ERR_INVALID_ARG;
  plan->use_graphs = on != 0;
  invalidate_graph(plan);
  return FDI_OK;
}

}  // extern "C"
