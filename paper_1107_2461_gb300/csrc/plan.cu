// Plan creation and the small C-ABI entry points (status, options, results).
//
// A plan holds, per direction and per unknown kind, the 1D finite-volume
// operator D = M^{-1} K (Sec. 3, Eq. 23) and its eigen decomposition
// D = E Lambda E^{-1} (Eq. 24), computed once per grid (Sec. 3: O(n^3), "its
// computational cost can be neglected") and kept resident on the device.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include <utility>

#include "fdi_internal.h"

namespace fdi {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

// Status of a finished solve from its device record and the plan's wait-limit
// flag: a kernel that gave up waiting, a non-finite right-hand side, a
// numerical failure, or a residual above the tolerance of that solve.
fdi_status solve_status(const fdi_plan* plan, const DevStatus& st, int kerr) {
  if (kerr) {
    set_error("a tensor-core kernel stopped at a wait limit");
    return FDI_ERR_TIMEOUT;
  }
  if (st.error == 7) {
    set_error("non-finite values in the right-hand side");
    return FDI_ERR_INVALID_ARG;
  }
  if (st.error) {
    set_error("numerical breakdown (non-finite residual, Krylov breakdown or iteration limit)");
    return FDI_ERR_NOT_CONVERGED;
  }
  if (!(st.rel_res <= (st.tol_used > 0.0 ? st.tol_used : plan->tol))) {
    set_error("residual above the tolerance after the last refinement step");
    return FDI_ERR_NOT_CONVERGED;
  }
  return FDI_OK;
}

static cudaEvent_t pool_event(fdi_plan* p) {
  cudaEvent_t e = nullptr;
  if (!p->event_pool.empty()) {
    e = p->event_pool.back();
    p->event_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    e = nullptr;
  }
  return e;
}

KTimer::KTimer(fdi_plan* p_, const char* name_, cudaStream_t s_) : p(p_), name(name_), s(s_) {
  if (p && p->timing) {
    e0 = pool_event(p);
    if (e0) cudaEventRecord(e0, s);
  }
}

KTimer::~KTimer() {
  if (p && p->timing && e0) {
    cudaEvent_t e1 = pool_event(p);
    if (e1) {
      cudaEventRecord(e1, s);
      p->pending.push_back({name, e0, e1});
    } else {
      p->event_pool.push_back(e0);
    }
  }
}

namespace {

// Cell-centred operator (n unknowns): interior flux 1/(c_{i+1}-c_i); a
// Dirichlet wall adds the flux to the wall value 0 at half a cell, 2/h.
void cell_op(const double* x, int n, int bc_lo, int bc_hi, std::vector<double>& m,
             std::vector<double>& kd, std::vector<double>& ko) {
  m.assign(n, 0.0);
  kd.assign(n, 0.0);
  ko.assign(n, 0.0);
  for (int i = 0; i < n; ++i) m[i] = x[i + 1] - x[i];
  for (int i = 0; i + 1 < n; ++i) {
    double ci = 0.5 * (x[i] + x[i + 1]), cj = 0.5 * (x[i + 1] + x[i + 2]);
    double g = 1.0 / (cj - ci);
    ko[i] = g;
    kd[i] -= g;
    kd[i + 1] -= g;
  }
  if (bc_lo == FDI_BC_DIRICHLET) kd[0] -= 2.0 / m[0];
  if (bc_hi == FDI_BC_DIRICHLET) kd[n - 1] -= 2.0 / m[n - 1];
}

// Face operator (n-1 unknowns on the interior faces, walls u = 0): flux
// coefficient 1/h_i across cell i, control volume c_j - c_{j-1}.
void face_op(const double* x, int n, std::vector<double>& m, std::vector<double>& kd,
             std::vector<double>& ko) {
  int u = n - 1;
  m.assign(u, 0.0);
  kd.assign(u, 0.0);
  ko.assign(u, 0.0);
  for (int j = 1; j < n; ++j) {
    double cl = 0.5 * (x[j - 1] + x[j]), cr = 0.5 * (x[j] + x[j + 1]);
    m[j - 1] = cr - cl;
  }
  for (int i = 0; i < n; ++i) {
    double g = 1.0 / (x[i + 1] - x[i]);
    int a = i - 1, b = i;  // unknown indices of faces i and i+1
    if (a >= 0 && a < u) kd[a] -= g;
    if (b >= 0 && b < u) kd[b] -= g;
    if (a >= 0 && b < u) ko[a] = g;
  }
}

template <typename T>
fdi_status dev_alloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? FDI_ERR_OUT_OF_MEMORY : FDI_ERR_CUDA;
  }
  return FDI_OK;
}

#define FDI_TRY(expr)                 \
  do {                                \
    fdi_status _s = (expr);           \
    if (_s != FDI_OK) return _s;      \
  } while (0)

fdi_status make_axis(Axis** out, const std::vector<double>& m, const std::vector<double>& kd,
                     const std::vector<double>& ko, bool zero_flux, cudaStream_t s) {
  Axis* ax = new Axis();
  *out = ax;
  int n = (int)m.size();
  ax->n = n;
  ax->zero_flux = zero_flux;
  ax->h_m = m;
  ax->h_kd = kd;
  ax->h_ko = ko;
  std::vector<double> wp(n, 0.0), wm(n, 0.0), w0(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double kp = (i + 1 < n) ? ko[i] : 0.0;
    double km = (i > 0) ? ko[i - 1] : 0.0;
    wp[i] = kp / m[i];
    wm[i] = km / m[i];
    // wall term: nonzero only in the first and last cell (interior cells have none)
    w0[i] = (i == 0 || i == n - 1) ? (kd[i] + kp + km) / m[i] : 0.0;
  }
  FDI_TRY(dev_alloc(&ax->m, n));
  FDI_TRY(dev_alloc(&ax->kd, n));
  FDI_TRY(dev_alloc(&ax->ko, n));
  FDI_TRY(dev_alloc(&ax->wp, n));
  FDI_TRY(dev_alloc(&ax->wm, n));
  FDI_TRY(dev_alloc(&ax->w0, n));
  FDI_TRY(dev_alloc(&ax->lam, n));
  FDI_TRY(dev_alloc(&ax->E, (size_t)n * n));
  FDI_TRY(dev_alloc(&ax->Einv, (size_t)n * n));
  FDI_CUDA_TRY(cudaMemcpyAsync(ax->m, m.data(), n * 8, cudaMemcpyHostToDevice, s));
  FDI_CUDA_TRY(cudaMemcpyAsync(ax->kd, kd.data(), n * 8, cudaMemcpyHostToDevice, s));
  FDI_CUDA_TRY(cudaMemcpyAsync(ax->ko, ko.data(), n * 8, cudaMemcpyHostToDevice, s));
  FDI_CUDA_TRY(cudaMemcpyAsync(ax->wp, wp.data(), n * 8, cudaMemcpyHostToDevice, s));
  FDI_CUDA_TRY(cudaMemcpyAsync(ax->wm, wm.data(), n * 8, cudaMemcpyHostToDevice, s));
  FDI_CUDA_TRY(cudaMemcpyAsync(ax->w0, w0.data(), n * 8, cudaMemcpyHostToDevice, s));
  // the host vectors must outlive the async copies: synchronise before returning
  FDI_CUDA_TRY(cudaStreamSynchronize(s));
  return FDI_OK;
}

void free_axis(Axis* ax) {
  if (!ax) return;
  mixed_free_axis(ax);
  void* ptrs[] = {ax->m, ax->kd, ax->ko, ax->wp, ax->wm, ax->w0, ax->lam, ax->E, ax->Einv};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete ax;
}

}  // namespace

void swap_slot(fdi_plan* p, fdi_work_slot& w) {
  for (int i = 0; i < 5; ++i) std::swap(p->ws[i], w.ws[i]);
  for (int i = 0; i < 4; ++i) std::swap(p->wf[i], w.wf[i]);
  std::swap(p->xdf, w.xdf);
  std::swap(p->wr1, w.wr1);
  std::swap(p->wr1_plane, w.wr1_plane);
  std::swap(p->d_scales, w.d_scales);
  std::swap(p->lam_w, w.lam_w);
  std::swap(p->partials, w.partials);
  std::swap(p->d_status, w.d_status);
  std::swap(p->d_counter, w.d_counter);
}

fdi_status alloc_workspace(fdi_plan* p) {
  for (int i = 0; i < 5; ++i) FDI_TRY(dev_alloc(&p->ws[i], (size_t)p->Pmax));
  FDI_TRY(dev_alloc(&p->partials, (size_t)p->npartials * 4));
  FDI_TRY(dev_alloc(&p->d_status, 1));
  FDI_CUDA_TRY(cudaMemset(p->d_status, 0, sizeof(DevStatus)));
  return FDI_OK;
}

void free_workspace(fdi_plan* p) {
  for (double*& w : p->ws) {
    if (w) cudaFree(w);
    w = nullptr;
  }
  for (float*& w : p->wf) {
    if (w) cudaFree(w);
    w = nullptr;
  }
  void* ptrs[] = {p->xdf, p->wr1, p->d_counter, p->d_scales, p->lam_w, p->partials, p->d_status};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  p->xdf = nullptr;
  p->wr1 = nullptr;
  p->d_counter = nullptr;
  p->d_scales = nullptr;
  p->lam_w = nullptr;
  p->partials = nullptr;
  p->d_status = nullptr;
}

namespace {

void free_plan(fdi_plan* p) {
  if (!p) return;
  invalidate_graph(p);
  free_host_staging(p);
  for (double*& t : p->tstage) {
    if (t) cudaFree(t);
    t = nullptr;
  }
  for (auto& t : p->pending) {
    cudaEventDestroy(t.e0);
    cudaEventDestroy(t.e1);
  }
  for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
  for (Axis* a : p->axes) free_axis(a);
  for (int c = 0; c < 3; ++c) {
    swap_slot(p, p->extra[c]);
    free_workspace(p);
    swap_slot(p, p->extra[c]);
    if (p->sstream[c]) cudaStreamDestroy(p->sstream[c]);
    if (p->sjoin[c]) cudaEventDestroy(p->sjoin[c]);
  }
  if (p->sfork) cudaEventDestroy(p->sfork);
  if (p->cstream) cudaStreamDestroy(p->cstream);
  free_workspace(p);
  for (double* w : p->sk)
    if (w) cudaFree(w);
  for (double* w : p->skf)
    if (w) cudaFree(w);
  for (int d = 0; d < 3; ++d) {
    if (p->mac_ih[d]) cudaFree(p->mac_ih[d]);
    if (p->mac_idc[d]) cudaFree(p->mac_idc[d]);
  }
  if (p->d_kry) cudaFree(p->d_kry);
  if (p->kpartials) cudaFree(p->kpartials);
  if (p->d_err) cudaFree(p->d_err);
  if (p->h_flag) cudaFreeHost(p->h_flag);
  delete p;
}

fdi_status build_plan(fdi_plan* p, const double* const faces[3], const fdi_bc bc_lo[3],
                      const fdi_bc bc_hi[3], cudaStream_t s) {
  int* d_err = nullptr;
  FDI_TRY(dev_alloc(&d_err, 1));
  FDI_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  std::vector<double> m, kd, ko;
  fdi_status st = FDI_OK;
  if (p->grid == FDI_GRID_CELL) {
    Axis* ax[3];
    for (int d = 0; d < 3 && st == FDI_OK; ++d) {
      cell_op(faces[d], p->n[d], bc_lo[d], bc_hi[d], m, kd, ko);
      bool zf = bc_lo[d] == FDI_BC_NEUMANN && bc_hi[d] == FDI_BC_NEUMANN;
      st = make_axis(&ax[d], m, kd, ko, zf, s);
      p->axes.push_back(ax[d]);
    }
    if (st == FDI_OK) {
      Field& f = p->fields[0];
      for (int d = 0; d < 3; ++d) {
        f.ax[d] = ax[d];
        f.n[d] = ax[d]->n;
      }
    }
    p->nfields = 1;
  } else {
    // per direction: cell-Dirichlet, face, cell-Neumann
    Axis* cd[3];
    Axis* fc[3];
    Axis* cn[3];
    for (int d = 0; d < 3 && st == FDI_OK; ++d) {
      cell_op(faces[d], p->n[d], FDI_BC_DIRICHLET, FDI_BC_DIRICHLET, m, kd, ko);
      st = make_axis(&cd[d], m, kd, ko, false, s);
      p->axes.push_back(cd[d]);
      if (st != FDI_OK) break;
      face_op(faces[d], p->n[d], m, kd, ko);
      st = make_axis(&fc[d], m, kd, ko, false, s);
      p->axes.push_back(fc[d]);
      if (st != FDI_OK) break;
      cell_op(faces[d], p->n[d], FDI_BC_NEUMANN, FDI_BC_NEUMANN, m, kd, ko);
      st = make_axis(&cn[d], m, kd, ko, true, s);
      p->axes.push_back(cn[d]);
    }
    if (st == FDI_OK) {
      for (int d = 0; d < 3; ++d) p->fields[0].ax[d] = cn[d];
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) p->fields[1 + c].ax[d] = (d == c) ? fc[d] : cd[d];
      for (int fi = 0; fi < 4; ++fi)
        for (int d = 0; d < 3; ++d) p->fields[fi].n[d] = p->fields[fi].ax[d]->n;
    }
    p->nfields = 4;
  }
  int h_err = 0;
  if (st == FDI_OK) st = eigen_decompose_all(p->axes, s, d_err);
  if (st == FDI_OK) {
    cudaError_t e = cudaMemcpy(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      set_error(std::string("eigen status copy: ") + cudaGetErrorString(e));
      st = FDI_ERR_CUDA;
    } else if (h_err != 0) {
      set_error("plan eigen decomposition did not converge");
      st = FDI_ERR_NOT_CONVERGED;
    }
  }
  cudaFree(d_err);
  if (st != FDI_OK) return st;
  for (int fi = 0; fi < p->nfields; ++fi) {
    Field& f = p->fields[fi];
    f.P = (long long)f.n[0] * f.n[1] * f.n[2];
    double vx = 0, vy = 0, vz = 0;
    for (double v : f.ax[0]->h_m) vx += v;
    for (double v : f.ax[1]->h_m) vy += v;
    for (double v : f.ax[2]->h_m) vz += v;
    f.vol_sum = vx * vy * vz;
    f.zero_flux_all = f.ax[0]->zero_flux && f.ax[1]->zero_flux && f.ax[2]->zero_flux;
    if (f.P > p->Pmax) p->Pmax = f.P;
  }
  p->npartials = 16384;  // per-block partial sums of the reductions (>= blocks of any reduction grid)
  FDI_TRY(alloc_workspace(p));
  FDI_CUDA_TRY(cudaMallocHost((void**)&p->h_flag, sizeof(int) * 4));
  if (p->prec != FDI_PREC_FP64) FDI_TRY(mixed_setup(p));
  if (p->grid == FDI_GRID_MAC) {
    FDI_TRY(stokes_setup(p));
    // three more workspaces and streams for the concurrent velocity solves
    for (int c = 0; c < 3; ++c) {
      swap_slot(p, p->extra[c]);
      fdi_status st2 = alloc_workspace(p);
      if (st2 == FDI_OK && p->prec != FDI_PREC_FP64) st2 = mixed_alloc_workspace(p);
      swap_slot(p, p->extra[c]);
      p->nextra = c + 1;
      FDI_TRY(st2);
      FDI_CUDA_TRY(cudaStreamCreateWithFlags(&p->sstream[c], cudaStreamNonBlocking));
      FDI_CUDA_TRY(cudaEventCreateWithFlags(&p->sjoin[c], cudaEventDisableTiming));
    }
    FDI_CUDA_TRY(cudaEventCreateWithFlags(&p->sfork, cudaEventDisableTiming));
  }
  return FDI_OK;
}

}  // namespace
}  // namespace fdi

using namespace fdi;

extern "C" {

const char* fdi_status_string(fdi_status s) {
  switch (s) {
    case FDI_OK: return "FDI_OK";
    case FDI_ERR_INVALID_ARG: return "FDI_ERR_INVALID_ARG";
    case FDI_ERR_OUT_OF_MEMORY: return "FDI_ERR_OUT_OF_MEMORY";
    case FDI_ERR_CUDA: return "FDI_ERR_CUDA";
    case FDI_ERR_NOT_CONVERGED: return "FDI_ERR_NOT_CONVERGED";
    case FDI_ERR_TIMEOUT: return "FDI_ERR_TIMEOUT";
    case FDI_ERR_SINGULAR: return "FDI_ERR_SINGULAR";
    case FDI_ERR_UNSUPPORTED: return "FDI_ERR_UNSUPPORTED";
  }
  return "FDI_ERR_UNKNOWN";
}

const char* fdi_last_error_message(void) { return g_last_error.c_str(); }

fdi_status fdi_plan_create(const double* const faces[3], const int n[3], const fdi_bc bc_lo[3],
                           const fdi_bc bc_hi[3], fdi_grid grid, fdi_precision prec, int thomas_axis,
                           fdi_plan** out) {
  if (!out) return FDI_ERR_INVALID_ARG;
  *out = nullptr;
  if (!faces || !n) return FDI_ERR_INVALID_ARG;
  if (grid != FDI_GRID_CELL && grid != FDI_GRID_MAC) return FDI_ERR_INVALID_ARG;
  if (prec < FDI_PREC_FP64 || prec > FDI_PREC_MIXED_F16) return FDI_ERR_INVALID_ARG;
  if (prec == FDI_PREC_MIXED_TF32 || prec == FDI_PREC_MIXED_BF16) {
    set_error("fdi_plan_create: FDI_PREC_MIXED_TF32 and FDI_PREC_MIXED_BF16 are not built; use FDI_PREC_MIXED_F16");
    return FDI_ERR_UNSUPPORTED;
  }
  if (grid == FDI_GRID_CELL && (!bc_lo || !bc_hi)) return FDI_ERR_INVALID_ARG;
  if (thomas_axis < -2 || thomas_axis > 2) {
    set_error("thomas_axis must be 0, 1, 2 (Thomas along x, y, z), -2 (the longest direction) or -1 (TPF)");
    return FDI_ERR_UNSUPPORTED;
  }
  if (thomas_axis == -2) {
    // the direction with the most cells (Sec. 3); ties go to z, then y
    thomas_axis = 2;
    if (n[1] > n[thomas_axis]) thomas_axis = 1;
    if (n[0] > n[thomas_axis]) thomas_axis = 0;
  }
  if (grid == FDI_GRID_MAC && thomas_axis != 2 && thomas_axis != -1) {
    set_error("a staggered (MAC) plan runs its Thomas sweeps along z (thomas_axis 2 or -1)");
    return FDI_ERR_UNSUPPORTED;
  }
  for (int d = 0; d < 3; ++d) {
    if (!faces[d] || n[d] < 2 || n[d] > kMaxN) {
      set_error("each direction needs 2 <= n <= 256 cells and a face array");
      return FDI_ERR_INVALID_ARG;
    }
    if (grid == FDI_GRID_MAC && n[d] < 3) {
      set_error("a staggered grid needs n >= 3 cells per direction");
      return FDI_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n[d]; ++i)
      if (!(faces[d][i + 1] > faces[d][i]) || !std::isfinite(faces[d][i + 1]) ||
          !std::isfinite(faces[d][i])) {
        set_error("faces must be finite and strictly ascending");
        return FDI_ERR_INVALID_ARG;
      }
    if (grid == FDI_GRID_CELL && ((unsigned)bc_lo[d] > 1u || (unsigned)bc_hi[d] > 1u))
      return FDI_ERR_INVALID_ARG;
  }
  fdi_plan* p = new fdi_plan();
  p->grid = grid;
  p->prec = prec;
  // Thomas along x or y: the plan is built on the grid with that axis moved to
  // z (internal axis d is external axis perm[d])
  p->thomas_ext = thomas_axis;
  if (thomas_axis == 0) {
    p->perm[0] = 2;
    p->perm[2] = 0;
  } else if (thomas_axis == 1) {
    p->perm[1] = 2;
    p->perm[2] = 1;
  }
  p->thomas_axis = thomas_axis == -1 ? -1 : 2;
  const double* faces_i[3];
  int n_i[3];
  fdi_bc lo_i[3] = {FDI_BC_DIRICHLET, FDI_BC_DIRICHLET, FDI_BC_DIRICHLET};
  fdi_bc hi_i[3] = {FDI_BC_DIRICHLET, FDI_BC_DIRICHLET, FDI_BC_DIRICHLET};
  for (int d = 0; d < 3; ++d) {
    faces_i[d] = faces[p->perm[d]];
    n_i[d] = n[p->perm[d]];
    if (bc_lo) lo_i[d] = bc_lo[p->perm[d]];
    if (bc_hi) hi_i[d] = bc_hi[p->perm[d]];
    p->n[d] = n_i[d];
    p->n_ext[d] = n[d];
  }
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    delete p;
    set_error("no CUDA device");
    return FDI_ERR_CUDA;
  }
  if (prec == FDI_PREC_FP64) {
    p->tol = 1e-11;
    p->max_refine = 2;
    p->ktol = 1e-11;
  } else {
    p->tol = 1e-10;
    p->max_refine = 3;
    p->ktol = 1e-10;
  }
  cudaStream_t s;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    delete p;
    set_error("stream creation failed");
    return FDI_ERR_CUDA;
  }
  fdi_status st = build_plan(p, faces_i, lo_i, hi_i, s);
  if (st == FDI_OK && (thomas_axis == 0 || thomas_axis == 1)) {
    const size_t P = (size_t)n[0] * n[1] * n[2];
    for (double*& t : p->tstage) {
      if (cudaMalloc(&t, P * sizeof(double)) != cudaSuccess) {
        set_error("cudaMalloc of the permuted staging fields failed");
        st = FDI_ERR_OUT_OF_MEMORY;
        break;
      }
    }
  }
  cudaError_t e = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (st == FDI_OK && e != cudaSuccess) {
    set_error(std::string("plan creation: ") + cudaGetErrorString(e));
    st = FDI_ERR_CUDA;
  }
  if (st != FDI_OK) {
    cudaDeviceSynchronize();
    free_plan(p);
    return st;
  }
  apply_tuning(p);  // a configuration autotuned earlier for this grid shape
  *out = p;
  return FDI_OK;
}

fdi_status fdi_plan_destroy(fdi_plan* plan) {
  if (!plan) return FDI_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  free_plan(plan);
  return FDI_OK;
}

fdi_status fdi_plan_set_tolerances(fdi_plan* plan, double tol, int max_refine, double krylov_tol,
                                   int max_iters) {
  if (!plan || !(tol > 0) || max_refine < 0 || max_refine > kMaxRefineCap || !(krylov_tol > 0) ||
      max_iters < 1)
    return FDI_ERR_INVALID_ARG;
  plan->tol = tol;
  invalidate_graph(plan);
  plan->max_refine = max_refine;
  plan->ktol = krylov_tol;
  plan->kmaxit = max_iters;
  return FDI_OK;
}

fdi_status fdi_last_result(const fdi_plan* plan, int* iters, int* refine_steps, double* rel_residual) {
  if (!plan) return FDI_ERR_INVALID_ARG;
  DevStatus st;
  cudaError_t e = cudaMemcpy(&st, plan->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    set_error(std::string("status copy: ") + cudaGetErrorString(e));
    return FDI_ERR_CUDA;
  }
  if (iters) *iters = st.iters;
  if (refine_steps) *refine_steps = st.refine_steps;
  if (rel_residual) *rel_residual = st.rel_res;
  int kerr = 0;
  if (plan->d_err) {
    e = cudaMemcpy(&kerr, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      set_error(std::string("status copy: ") + cudaGetErrorString(e));
      return FDI_ERR_CUDA;
    }
  }
  return fdi::solve_status(plan, st, kerr);
}

fdi_status fdi_plan_eigen(const fdi_plan* plan, fdi_field field, int d, double* lam, double* E,
                          double* Einv, int* m) {
  if (!plan || d < 0 || d > 2 || (int)field < 0 || (int)field >= plan->nfields) return FDI_ERR_INVALID_ARG;
  int di = d;  // internal axis holding external direction d
  for (int q = 0; q < 3; ++q)
    if (plan->perm[q] == d) di = q;
  const Axis* ax = plan->fields[(int)field].ax[di];
  int n = ax->n;
  if (m) *m = n;
  if (lam) FDI_CUDA_TRY(cudaMemcpy(lam, ax->lam, n * 8, cudaMemcpyDeviceToHost));
  if (E) FDI_CUDA_TRY(cudaMemcpy(E, ax->E, (size_t)n * n * 8, cudaMemcpyDeviceToHost));
  if (Einv) FDI_CUDA_TRY(cudaMemcpy(Einv, ax->Einv, (size_t)n * n * 8, cudaMemcpyDeviceToHost));
  return FDI_OK;
}

fdi_status fdi_plan_enable_timing(fdi_plan* plan, int on) {
  if (!plan) return FDI_ERR_INVALID_ARG;
  plan->timing = on != 0;
  return FDI_OK;
}

fdi_status fdi_plan_kernel_times(fdi_plan* plan, int max, const char** names, double* total_ms,
                                 long long* launches, int* count) {
  if (!plan || max < 0 || !count) return FDI_ERR_INVALID_ARG;
  for (auto& t : plan->pending) {
    FDI_CUDA_TRY(cudaEventSynchronize(t.e1));
    float ms = 0.f;
    FDI_CUDA_TRY(cudaEventElapsedTime(&ms, t.e0, t.e1));
    bool found = false;
    for (auto& k : plan->ktimes)
      if (k.name == t.name) {
        k.ms += ms;
        k.n += 1;
        found = true;
        break;
      }
    if (!found) plan->ktimes.push_back({t.name, (double)ms, 1});
    plan->event_pool.push_back(t.e0);
    plan->event_pool.push_back(t.e1);
  }
  plan->pending.clear();
  int c = 0;
  for (auto& k : plan->ktimes) {
    if (c >= max) break;
    if (names) names[c] = k.name.c_str();
    if (total_ms) total_ms[c] = k.ms;
    if (launches) launches[c] = k.n;
    ++c;
  }
  *count = c;
  return FDI_OK;
}

fdi_status fdi_plan_reset_kernel_times(fdi_plan* plan) {
  if (!plan) return FDI_ERR_INVALID_ARG;
  int c = 0;
  fdi_status st = fdi_plan_kernel_times(plan, 0, nullptr, nullptr, nullptr, &c);
  plan->ktimes.clear();
  return st;
}

fdi_status fdi_last_launch_count(const fdi_plan* plan, long long* launches) {
  if (!plan || !launches) return FDI_ERR_INVALID_ARG;
  *launches = plan->launches + fdi::stokes_loop_launches(plan);
  return FDI_OK;
}

}  // extern "C"
