// Serving runtime: a request loop for Stokes-inverse applications (the calls a
// time-stepper-based Newton or Arnoldi iteration issues, Sec. 1-2) with uneven
// grids and differing dt / Re.
//
//   * Plans (1D operators, eigenbases, workspaces) stay resident on the device
//     in a cache keyed by (grid, stretching, precision); idle plans are evicted
//     least-recently-used when memory is needed.
//   * Admission by device-memory footprint: a request is started only when its
//     plan (cached or new) and its fields fit in the budget.  Strict FIFO, so a
//     large request is never overtaken indefinitely.
//   * Continuous batching: `slots` worker threads, each with its own CUDA
//     stream; a request arriving while others run is admitted as soon as a
//     slot and memory are free, and its kernels overlap theirs on the device.
//   * Each worker runs the whole request: host -> device copies of the forcing,
//     the Stokes inverse on its plan (pressure system by conjugate gradients in
//     the volume-weighted inner product), device -> host copies of u and p.  A plan
//     is used by one request at a time (plans are not shared across streams).
//   * Latency = completion - submission (queueing included); p50 / p99 and
//     throughput are reported by fdi_server_stats.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <vector>

#include "fdi_internal.h"

using fdi::set_error;

namespace {

using Clock = std::chrono::steady_clock;

struct PlanKey {
  int n0, n1, n2;
  double beta;
  int prec;
  bool operator<(const PlanKey& o) const {
    return std::tie(n0, n1, n2, beta, prec) < std::tie(o.n0, o.n1, o.n2, o.beta, o.prec);
  }
};

struct PlanEntry {
  fdi_plan* plan = nullptr;
  size_t bytes = 0;
  bool busy = false;
  long long last_use = 0;
};

struct Request {
  long long ticket = 0;
  fdi_stokes_request req{};
  Clock::time_point t_submit, t_start, t_done;
  int state = 0;  // 0 queued, 1 running, 2 done
  fdi_status status = FDI_OK;
  int iters = 0;
  double rel = 0.0;
  size_t field_bytes = 0;
};

long long cells(const int n[3]) { return (long long)n[0] * n[1] * n[2]; }

// Field sizes of a MAC request: u, v, w on interior faces, p at cells.
void mac_sizes(const int n[3], long long sz[4]) {
  sz[0] = (long long)(n[0] - 1) * n[1] * n[2];
  sz[1] = (long long)n[0] * (n[1] - 1) * n[2];
  sz[2] = (long long)n[0] * n[1] * (n[2] - 1);
  sz[3] = cells(n);
}

// Faces of one direction: x_i = (1 + tanh(beta (2 i / n - 1)) / tanh(beta)) / 2,
// uniform for beta = 0.
std::vector<double> tanh_faces(int n, double beta) {
  std::vector<double> x(n + 1);
  for (int i = 0; i <= n; ++i) {
    const double s = 2.0 * i / n - 1.0;
    x[i] = beta > 0.0 ? 0.5 * (1.0 + std::tanh(beta * s) / std::tanh(beta)) : 0.5 * (1.0 + s);
  }
  x[0] = 0.0;
  x[n] = 1.0;
  return x;
}

}  // namespace

// Device bytes a MAC Stokes plan allocates (upper estimate of plan.cu,
// mixed.cu, tc_transform.cu and stokes.cu): per direction and kind the FP64
// operator and eigen data (+ split fp16 copies for mixed plans), four per-solve
// workspaces (five FP64 fields, partials, the mixed FP32 planes), and the
// Krylov / face vectors.
extern "C" size_t fdi_stokes_plan_bytes_estimate(const int n[3], int prec) {
  const long long P = cells(n);
  size_t b = 0;
  for (int d = 0; d < 3; ++d) {
    const size_t nd = (size_t)n[d] + 1;
    const size_t per_axis = 2 * nd * nd * 8 + 8 * nd * 8 + (prec != FDI_PREC_FP64 ? 2 * 2 * 2 * (nd + 32) * (nd + 32) * 2 : 0);
    b += 3 * per_axis;  // cell-Dirichlet, cell-Neumann, face kinds
  }
  const size_t Pp = (size_t)(n[0] + 4) * (n[1] + 4) * n[2];  // padded FP32 rows
  // four per-solve workspaces (the plan's own and one per velocity component)
  size_t slot = 5 * (size_t)P * 8 + (size_t)16384 * 4 * 8;  // FP64 workspace, partials
  if (prec == FDI_PREC_FP64) slot += 2 * (size_t)P * 8;      // Thomas factor cache
  if (prec != FDI_PREC_FP64) slot += 4 * Pp * 4 + 3 * (size_t)P * 4 + 2 * Pp * 4;
  b += 4 * slot;
  b += 11 * (size_t)P * 8 + 6 * (size_t)P * 8;  // Krylov vectors, cell volumes, face work fields
  b += (size_t)4 << 20;                          // small tables, slack
  return b;
}

struct fdi_server {
  size_t budget = 0, in_use = 0, peak = 0;
  int slots = 1;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv, cv_done;
  std::deque<Request*> queue;
  std::map<long long, Request*> all;
  std::map<PlanKey, std::vector<PlanEntry>> plans;
  std::vector<std::thread> workers;
  std::vector<double> latencies_ms;
  Clock::time_point first_submit, last_done;
  bool any = false, stop = false;
  long long next_ticket = 1, tick = 0, running = 0;
  long long plans_created = 0, plans_evicted = 0;
  fdi_status worker_error = FDI_OK;
};

namespace {

size_t request_field_bytes(const fdi_stokes_request& r) {
  long long sz[4];
  mac_sizes(r.n, sz);
  return (size_t)(2 * (sz[0] + sz[1] + sz[2]) + sz[3]) * sizeof(double);
}

// Under the lock: find an idle cached plan for the request or make room for a
// new one.  Returns the entry (existing) or nullptr with *need_new set when a
// plan must be created (its bytes are then already reserved); false when the
// request does not fit yet.
bool try_admit(fdi_server* sv, Request* rq, PlanEntry** entry, bool* need_new, size_t* plan_bytes) {
  const fdi_stokes_request& r = rq->req;
  const PlanKey key{r.n[0], r.n[1], r.n[2], r.beta, (int)r.prec};
  const size_t fb = request_field_bytes(r);
  *entry = nullptr;
  *need_new = false;
  auto it = sv->plans.find(key);
  if (it != sv->plans.end())
    for (PlanEntry& e : it->second)
      if (!e.busy) {
        if (sv->in_use + fb > sv->budget) return false;
        *entry = &e;
        return true;
      }
  const size_t pb = fdi_stokes_plan_bytes_estimate(r.n, (int)r.prec);
  // evict idle plans (least recently used first) until the request fits
  while (sv->in_use + pb + fb > sv->budget) {
    PlanEntry* victim = nullptr;
    PlanKey vkey{};
    for (auto& kv : sv->plans)
      for (PlanEntry& e : kv.second)
        if (!e.busy && (!victim || e.last_use < victim->last_use)) {
          victim = &e;
          vkey = kv.first;
        }
    if (!victim) return false;
    fdi_plan_destroy(victim->plan);
    sv->in_use -= victim->bytes;
    sv->plans_evicted += 1;
    auto& vec = sv->plans[vkey];
    vec.erase(vec.begin() + (victim - vec.data()));
    if (vec.empty()) sv->plans.erase(vkey);
  }
  *need_new = true;
  *plan_bytes = pb;
  return true;
}

// Requests up to this many cells run on a worker's high-priority stream: the
// GPU dispatches their blocks ahead of those of large requests running on
// other workers, so a small request's many short kernels are not queued behind
// a large solve's blocks (results are unaffected: the same launches run).
constexpr long long kHighPriorityCells = 128LL * 128 * 128;

void worker(fdi_server* sv) {
  cudaSetDevice(sv->device);
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  cudaStream_t s_lo = nullptr, s_hi = nullptr;
  if (cudaStreamCreateWithPriority(&s_lo, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
      cudaStreamCreateWithPriority(&s_hi, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->worker_error = FDI_ERR_CUDA;
    return;
  }
  for (;;) {
    Request* rq = nullptr;
    PlanEntry* entry = nullptr;
    fdi_plan* plan_in = nullptr;
    bool need_new = false;
    size_t pb = 0;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      for (;;) {
        if (sv->stop && sv->queue.empty()) break;
        if (!sv->queue.empty() && try_admit(sv, sv->queue.front(), &entry, &need_new, &pb)) {
          rq = sv->queue.front();
          sv->queue.pop_front();
          break;
        }
        sv->cv.wait(lk);
      }
      if (!rq) break;
      rq->field_bytes = request_field_bytes(rq->req);
      sv->in_use += rq->field_bytes + (need_new ? pb : 0);
      sv->peak = std::max(sv->peak, sv->in_use);
      if (entry) {
        entry->busy = true;
        entry->last_use = ++sv->tick;
        plan_in = entry->plan;  // entries may move when the cache grows
      }
      rq->state = 1;
      rq->t_start = Clock::now();
      sv->running += 1;
    }
    const fdi_stokes_request& r = rq->req;
    cudaStream_t s = cells(r.n) <= kHighPriorityCells ? s_hi : s_lo;
    fdi_status st = FDI_OK;
    fdi_plan* plan = plan_in;
    if (need_new) {
      std::vector<double> fx = tanh_faces(r.n[0], r.beta), fy = tanh_faces(r.n[1], r.beta),
                          fz = tanh_faces(r.n[2], r.beta);
      const double* faces[3] = {fx.data(), fy.data(), fz.data()};
      const fdi_bc dir[3] = {FDI_BC_DIRICHLET, FDI_BC_DIRICHLET, FDI_BC_DIRICHLET};
      st = fdi_plan_create(faces, r.n, dir, dir, FDI_GRID_MAC, r.prec, 2, &plan);
      // conjugate gradients in the volume-weighted inner product: one C-product
      // per iteration (the lowest latency of the three Krylov methods)
      if (st == FDI_OK && (st = fdi_plan_set_krylov(plan, 2)) != FDI_OK) {
        fdi_plan_destroy(plan);
        plan = nullptr;
      }
      std::lock_guard<std::mutex> lk(sv->mu);
      if (st == FDI_OK) {
        const PlanKey key{r.n[0], r.n[1], r.n[2], r.beta, (int)r.prec};
        PlanEntry e;
        e.plan = plan;
        e.bytes = pb;
        e.busy = true;
        e.last_use = ++sv->tick;
        sv->plans[key].push_back(e);
        sv->plans_created += 1;
      } else {
        sv->in_use -= pb;
      }
    }
    long long sz[4];
    mac_sizes(r.n, sz);
    double* dbuf = nullptr;
    if (st == FDI_OK) {
      if (cudaMallocAsync((void**)&dbuf, rq->field_bytes, s) != cudaSuccess) {
        set_error("server: request field allocation failed");
        st = FDI_ERR_OUT_OF_MEMORY;
      }
    }
    if (st == FDI_OK) {
      // device layout: f_u f_v f_w u_u u_v u_w p
      double* df[3] = {dbuf, dbuf + sz[0], dbuf + sz[0] + sz[1]};
      double* du[3] = {df[2] + sz[2], df[2] + sz[2] + sz[0], df[2] + sz[2] + sz[0] + sz[1]};
      double* dp = du[2] + sz[2];
      for (int c = 0; c < 3 && st == FDI_OK; ++c)
        if (cudaMemcpyAsync(df[c], r.f[c], sz[c] * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess)
          st = FDI_ERR_CUDA;
      const double* cf[3] = {df[0], df[1], df[2]};
      if (st == FDI_OK) st = fdi_stokes_solve(plan, r.dt, r.Re, cf, du, dp, (fdi_stream_t)s);
      for (int c = 0; c < 3 && st == FDI_OK; ++c)
        if (cudaMemcpyAsync(r.u[c], du[c], sz[c] * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
          st = FDI_ERR_CUDA;
      if (st == FDI_OK &&
          cudaMemcpyAsync(r.p, dp, sz[3] * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = FDI_ERR_CUDA;
      cudaFreeAsync(dbuf, s);
      if (cudaStreamSynchronize(s) != cudaSuccess && st == FDI_OK) st = FDI_ERR_CUDA;
    }
    int iters = 0, steps = 0;
    double rel = 0.0;
    if (st == FDI_OK) st = fdi_last_result(plan, &iters, &steps, &rel);
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->in_use -= rq->field_bytes;
      if (plan) {
        auto it = sv->plans.find(PlanKey{r.n[0], r.n[1], r.n[2], r.beta, (int)r.prec});
        if (it != sv->plans.end())
          for (PlanEntry& e : it->second)
            if (e.plan == plan) {
              e.busy = false;
              e.last_use = ++sv->tick;
            }
      }
      rq->status = st;
      rq->iters = iters;
      rq->rel = rel;
      rq->t_done = Clock::now();
      rq->state = 2;
      sv->running -= 1;
      sv->latencies_ms.push_back(std::chrono::duration<double, std::milli>(rq->t_done - rq->t_submit).count());
      sv->last_done = rq->t_done;
    }
    sv->cv.notify_all();
    sv->cv_done.notify_all();
  }
  cudaStreamDestroy(s_lo);
  cudaStreamDestroy(s_hi);
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const size_t i = std::min(v.size() - 1, (size_t)std::floor(q * (double)(v.size() - 1) + 0.5));
  return v[i];
}

}  // namespace

extern "C" {

fdi_status fdi_server_create(size_t hbm_budget_bytes, int slots, fdi_server** out) {
  if (!out || slots < 1 || slots > 64 || hbm_budget_bytes == 0) return FDI_ERR_INVALID_ARG;
  *out = nullptr;
  fdi_server* sv = new fdi_server();
  sv->budget = hbm_budget_bytes;
  sv->slots = slots;
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    set_error("server: no CUDA device");
    return FDI_ERR_CUDA;
  }
  for (int i = 0; i < slots; ++i) sv->workers.emplace_back(worker, sv);
  *out = sv;
  return FDI_OK;
}

fdi_status fdi_server_submit(fdi_server* sv, const fdi_stokes_request* req, long long* ticket) {
  if (!sv || !req || !ticket) return FDI_ERR_INVALID_ARG;
  for (int d = 0; d < 3; ++d)
    if (req->n[d] < 2 || req->n[d] > fdi::kMaxN || !req->f[d] || !req->u[d]) return FDI_ERR_INVALID_ARG;
  if (!req->p || !(req->dt > 0) || !(req->Re > 0) || !(req->beta >= 0) || !std::isfinite(req->dt) ||
      !std::isfinite(req->Re))
    return FDI_ERR_INVALID_ARG;
  if (req->prec != FDI_PREC_FP64 && req->prec != FDI_PREC_MIXED_F16) return FDI_ERR_UNSUPPORTED;
  const size_t need = fdi_stokes_plan_bytes_estimate(req->n, (int)req->prec) + request_field_bytes(*req);
  std::lock_guard<std::mutex> lk(sv->mu);
  if (need > sv->budget) {
    set_error("server: request footprint exceeds the device-memory budget");
    return FDI_ERR_OUT_OF_MEMORY;
  }
  Request* rq = new Request();
  rq->ticket = sv->next_ticket++;
  rq->req = *req;
  rq->t_submit = Clock::now();
  if (!sv->any) {
    sv->first_submit = rq->t_submit;
    sv->any = true;
  }
  sv->all[rq->ticket] = rq;
  sv->queue.push_back(rq);
  *ticket = rq->ticket;
  sv->cv.notify_all();
  return FDI_OK;
}

fdi_status fdi_server_poll(fdi_server* sv, long long ticket, int wait, fdi_stokes_result* res) {
  if (!sv || !res) return FDI_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) return FDI_ERR_INVALID_ARG;
  Request* rq = it->second;
  if (wait)
    sv->cv_done.wait(lk, [&] { return rq->state == 2 || sv->worker_error != FDI_OK; });
  res->state = rq->state;
  res->status = rq->status;
  res->iters = rq->iters;
  res->rel_residual = rq->rel;
  res->queue_ms = rq->state >= 1 ? std::chrono::duration<double, std::milli>(rq->t_start - rq->t_submit).count() : 0.0;
  res->latency_ms = rq->state == 2 ? std::chrono::duration<double, std::milli>(rq->t_done - rq->t_submit).count() : 0.0;
  return sv->worker_error;
}

fdi_status fdi_server_drain(fdi_server* sv) {
  if (!sv) return FDI_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  sv->cv_done.wait(lk, [&] { return (sv->queue.empty() && sv->running == 0) || sv->worker_error != FDI_OK; });
  return sv->worker_error;
}

fdi_status fdi_server_stats(fdi_server* sv, fdi_server_report* out) {
  if (!sv || !out) return FDI_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  out->completed = (long long)sv->latencies_ms.size();
  out->p50_ms = percentile(sv->latencies_ms, 0.50);
  out->p99_ms = percentile(sv->latencies_ms, 0.99);
  const double span =
      sv->any && out->completed > 0 ? std::chrono::duration<double>(sv->last_done - sv->first_submit).count() : 0.0;
  out->throughput_rps = span > 0 ? (double)out->completed / span : 0.0;
  out->peak_bytes = sv->peak;
  out->bytes_in_use = sv->in_use;
  out->plans_created = sv->plans_created;
  out->plans_evicted = sv->plans_evicted;
  long long cached = 0;
  for (auto& kv : sv->plans) cached += (long long)kv.second.size();
  out->plans_cached = cached;
  return FDI_OK;
}

fdi_status fdi_server_destroy(fdi_server* sv) {
  if (!sv) return FDI_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  for (std::thread& t : sv->workers) t.join();
  for (auto& kv : sv->plans)
    for (PlanEntry& e : kv.second) fdi_plan_destroy(e.plan);
  for (auto& kv : sv->all) delete kv.second;
  delete sv;
  return FDI_OK;
}

}  // extern "C"
