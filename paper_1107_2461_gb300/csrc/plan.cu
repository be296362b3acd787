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

// periodic: ko[n-1] couples the last cell with the first (the flux weights
// wrap around and there is no wall term)
fdi_status make_axis(Axis** out, const std::vector<double>& m, const std::vector<double>& kd,
                     const std::vector<double>& ko, bool zero_flux, cudaStream_t s, bool periodic = false) {
  Axis* ax = new Axis();
  *out = ax;
  int n = (int)m.size();
  ax->n = n;
  ax->zero_flux = zero_flux;
  ax->periodic = periodic;
  ax->h_m = m;
  ax->h_kd = kd;
  ax->h_ko = ko;
  std::vector<double> wp(n, 0.0), wm(n, 0.0), w0(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double kp = (i + 1 < n || periodic) ? ko[i] : 0.0;
    double km = (i > 0) ? ko[i - 1] : (periodic ? ko[n - 1] : 0.0);
    wp[i] = kp / m[i];
    wm[i] = km / m[i];
    // wall term: nonzero only in the first and last cell (interior cells have none)
    w0[i] = (!periodic && (i == 0 || i == n - 1)) ? (kd[i] + kp + km) / m[i] : 0.0;
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
  std::swap(p->tf, w.tf);
  std::swap(p->tf_q, w.tf_q);
}

fdi_status alloc_thomas_cache(fdi_plan* p, long long q) {
  if (p->tf && p->tf_q >= q) return FDI_OK;
  if (p->tf) cudaFree(p->tf);
  p->tf = nullptr;
  p->tf_q = 0;
  FDI_TRY(dev_alloc(&p->tf, (size_t)(2 * q + 4)));
  // an impossible key (lambda < 0): the first sweep computes the factors
  const double key[4] = {0.0, -1.0, -1.0, 0.0};
  FDI_CUDA_TRY(cudaMemcpy(p->tf + 2 * q, key, sizeof(key), cudaMemcpyHostToDevice));
  p->tf_q = q;
  return FDI_OK;
}

fdi_status alloc_workspace(fdi_plan* p) {
  for (int i = 0; i < 5; ++i) FDI_TRY(dev_alloc(&p->ws[i], (size_t)p->Pmax));
  FDI_TRY(dev_alloc(&p->partials, (size_t)p->npartials * 4));
  FDI_TRY(dev_alloc(&p->d_status, 1));
  FDI_CUDA_TRY(cudaMemset(p->d_status, 0, sizeof(DevStatus)));
  // FP64 TPT sweeps keep their line factors for repeated (sigma, lambda)
  if (p->prec == FDI_PREC_FP64 && p->thomas_axis == 2) FDI_TRY(alloc_thomas_cache(p, p->Pmax));
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
  void* ptrs[] = {p->xdf, p->wr1, p->d_counter, p->d_scales, p->lam_w, p->partials, p->d_status, p->tf};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  p->xdf = nullptr;
  p->wr1 = nullptr;
  p->d_counter = nullptr;
  p->d_scales = nullptr;
  p->lam_w = nullptr;
  p->partials = nullptr;
  p->d_status = nullptr;
  p->tf = nullptr;
  p->tf_q = 0;
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
  for (void* q : {(void*)p->cyl_wy, (void*)p->cyl_wres, (void*)p->cyl_wy_f, (void*)p->cyl_wres_df, (void*)p->cyl_Er,
                  (void*)p->cyl_Eri, (void*)p->cyl_lr})
    if (q) cudaFree(q);
  if (p->d_kry) cudaFree(p->d_kry);
  if (p->kpartials) cudaFree(p->kpartials);
  if (p->kticket) cudaFree(p->kticket);
  if (p->d_err) cudaFree(p->d_err);
  if (p->res_bar) cudaFree(p->res_bar);
  if (p->h_flag) cudaFreeHost(p->h_flag);
  delete p;
}

fdi_status check_eigen_flag(const int* d_err) {
  int h_err = 0;
  cudaError_t e = cudaMemcpy(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    set_error(std::string("eigen status copy: ") + cudaGetErrorString(e));
    return FDI_ERR_CUDA;
  }
  if (h_err != 0) {
    set_error("plan eigen decomposition did not converge");
    return FDI_ERR_NOT_CONVERGED;
  }
  return FDI_OK;
}

fdi_status finish_plan(fdi_plan* p, cudaStream_t s);

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
  if (st == FDI_OK) st = eigen_decompose_all(p->axes, s, d_err);
  if (st == FDI_OK) st = check_eigen_flag(d_err);
  cudaFree(d_err);
  if (st != FDI_OK) return st;
  return finish_plan(p, s);
}

// field sizes and volumes, workspaces, mixed-precision and Stokes set-up of a
// plan whose axes, fields and eigen data are in place
fdi_status finish_plan(fdi_plan* p, cudaStream_t s) {
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

// ---------------------------------------------------------------------------
// Cylindrical grids (Sec. 6, Eq. 41-46), finite-volume reading: cells
// (r_i, theta_j, z_k); radial faces rho_0 < ... < rho_n (rho_0 = 0: the axis,
// a face of zero area that no flux crosses), centres c_i, annular areas
// A_i = (rho_{i+1}^2 - rho_i^2) / 2 = h_i c_i; radial flux through rho_{i+1}
// rho_{i+1} (u_{i+1} - u_i) / (c_{i+1} - c_i); a Dirichlet wall at rho_0 > 0 or
// rho_n over half a cell.  So D_rr = diag(A)^{-1} K_r, and the 1/r^2 of Eq. 41
// becomes per radial cell g_i = h_i / (c_i A_i) (the arc flux of the cell over
// its volume).  theta: M uniform cells on the full circle, periodic.

void radial_op(const double* rho, int n, int bc_in, int bc_out, std::vector<double>& A, std::vector<double>& kd,
               std::vector<double>& ko, std::vector<double>& g) {
  A.assign(n, 0.0);
  kd.assign(n, 0.0);
  ko.assign(n, 0.0);
  g.assign(n, 0.0);
  std::vector<double> c(n);
  for (int i = 0; i < n; ++i) {
    const double h = rho[i + 1] - rho[i];
    c[i] = 0.5 * (rho[i] + rho[i + 1]);
    A[i] = h * c[i];
    g[i] = h / (c[i] * A[i]);
  }
  for (int i = 0; i + 1 < n; ++i) {
    const double w = rho[i + 1] / (c[i + 1] - c[i]);
    ko[i] = w;
    kd[i] -= w;
    kd[i + 1] -= w;
  }
  if (rho[0] > 0.0 && bc_in == FDI_BC_DIRICHLET) kd[0] -= rho[0] / (0.5 * (rho[1] - rho[0]));
  if (bc_out == FDI_BC_DIRICHLET) kd[n - 1] -= rho[n] / (0.5 * (rho[n] - rho[n - 1]));
}

// Eigenbasis of the periodic second difference on M uniform cells (h = 2 pi / M,
// D = K / h with K = circ(-2, 1, 1) / h), in closed form: the discrete Fourier
// modes cos(2 pi k j / M) and sin(2 pi k j / M), eigenvalue -(4 / h^2) sin^2(pi k / M),
// normalised so that E^T diag(h) E = I.  Column order: the constant mode, then
// (cos k, sin k) for k = 1 .. (M-1)/2, then the alternating mode k = M/2 for
// even M (eigenvalues descending from 0, like the tridiagonal decompositions).
void periodic_eigen(int M, std::vector<double>& lam, std::vector<double>& E, std::vector<double>& Einv) {
  const double pi = 3.14159265358979323846;
  const double h = 2.0 * pi / M;
  lam.assign(M, 0.0);
  E.assign((size_t)M * M, 0.0);
  Einv.assign((size_t)M * M, 0.0);
  auto column = [&](int q, int k, bool sine) {
    const double sk = std::sin(pi * k / M);
    lam[q] = -4.0 / (h * h) * sk * sk;
    const double norm = (k == 0 || 2 * k == M) ? 1.0 / std::sqrt(M * h) : std::sqrt(2.0 / (M * h));
    for (int j = 0; j < M; ++j) {
      const double ang = 2.0 * pi * (double)(((long long)k * j) % M) / M;  // reduced exactly
      E[(size_t)j * M + q] = norm * (sine ? std::sin(ang) : std::cos(ang));
    }
  };
  column(0, 0, false);
  for (int k = 1; 2 * k < M; ++k) {
    column(2 * k - 1, k, false);
    column(2 * k, k, true);
  }
  if (M % 2 == 0) column(M - 1, M / 2, false);
  for (int j = 0; j < M; ++j)
    for (int q = 0; q < M; ++q) Einv[(size_t)q * M + j] = E[(size_t)j * M + q] * h;
}

template <typename T>
fdi_status upload(T** dst, const std::vector<T>& v) {
  FDI_TRY(dev_alloc(dst, v.size()));
  FDI_CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return FDI_OK;
}

// Internal order [r][theta][z]: x = z, y = theta, z = r, so the Thomas sweeps
// run along r (Eq. 44) and the x / y eigen transforms along z and theta.
fdi_status build_cyl_plan(fdi_plan* p, const double* rho, int nr, int M, const double* zf, int nz, fdi_bc bc_r_in,
                          fdi_bc bc_r_out, fdi_bc bc_z_lo, fdi_bc bc_z_hi, cudaStream_t s) {
  std::vector<double> m, kd, ko;
  Axis* az = nullptr;
  Axis* at = nullptr;
  Axis* ar = nullptr;
  cell_op(zf, nz, bc_z_lo, bc_z_hi, m, kd, ko);
  FDI_TRY(make_axis(&az, m, kd, ko, bc_z_lo == FDI_BC_NEUMANN && bc_z_hi == FDI_BC_NEUMANN, s));
  p->axes.push_back(az);
  const double pi = 3.14159265358979323846;
  const double h = 2.0 * pi / M;
  m.assign(M, h);
  kd.assign(M, -2.0 / h);
  ko.assign(M, 1.0 / h);
  FDI_TRY(make_axis(&at, m, kd, ko, true, s, true));
  p->axes.push_back(at);
  std::vector<double> A, g;
  radial_op(rho, nr, bc_r_in, bc_r_out, A, kd, ko, g);
  const bool r_closed = (rho[0] == 0.0 || bc_r_in == FDI_BC_NEUMANN) && bc_r_out == FDI_BC_NEUMANN;
  FDI_TRY(make_axis(&ar, A, kd, ko, r_closed, s));
  p->axes.push_back(ar);
  Field& f = p->fields[0];
  f.ax[0] = az;
  f.ax[1] = at;
  f.ax[2] = ar;
  for (int d = 0; d < 3; ++d) f.n[d] = f.ax[d]->n;
  p->nfields = 1;
  // closed-form theta eigenbasis, then the tridiagonal ones on the GPU
  {
    std::vector<double> lam, E, Einv;
    periodic_eigen(M, lam, E, Einv);
    FDI_CUDA_TRY(cudaMemcpy(at->lam, lam.data(), M * sizeof(double), cudaMemcpyHostToDevice));
    FDI_CUDA_TRY(cudaMemcpy(at->E, E.data(), E.size() * sizeof(double), cudaMemcpyHostToDevice));
    FDI_CUDA_TRY(cudaMemcpy(at->Einv, Einv.data(), Einv.size() * sizeof(double), cudaMemcpyHostToDevice));
    // weights of the theta eigenvalue (Thomas) and of the theta flux (residual)
    std::vector<double> wy(nr), wres(nr);
    for (int i = 0; i < nr; ++i) {
      wy[i] = A[i] * g[i];
      wres[i] = g[i] / (h * h);
    }
    FDI_TRY(upload(&p->cyl_wy, wy));
    FDI_TRY(upload(&p->cyl_wres, wres));
    if (p->thomas_axis == -1) {
      // Eq. 45: per theta mode j, D_rr + lambda_th,j g = E_{r,j} Lambda E_{r,j}^{-1},
      // i.e. K_r + lambda_th,j diag(A g) with the same diag(A)
      std::vector<double> kd_all((size_t)M * nr);
      for (int q = 0; q < M; ++q)
        for (int i = 0; i < nr; ++i) kd_all[(size_t)q * nr + i] = kd[i] + lam[q] * A[i] * g[i];
      double* d_kd = nullptr;
      FDI_TRY(upload(&d_kd, kd_all));
      fdi_status st = dev_alloc(&p->cyl_lr, (size_t)M * nr);
      if (st == FDI_OK) st = dev_alloc(&p->cyl_Er, (size_t)M * nr * nr);
      if (st == FDI_OK) st = dev_alloc(&p->cyl_Eri, (size_t)M * nr * nr);
      int* d_err = nullptr;
      if (st == FDI_OK) st = dev_alloc(&d_err, 1);
      if (st == FDI_OK && cudaMemset(d_err, 0, sizeof(int)) != cudaSuccess) st = FDI_ERR_CUDA;
      if (st == FDI_OK)
        st = eigen_decompose_batch(M, nr, ar->m, d_kd, ar->ko, r_closed, p->cyl_lr, p->cyl_Er, p->cyl_Eri, s, d_err);
      if (st == FDI_OK) st = check_eigen_flag(d_err);
      if (d_err) cudaFree(d_err);
      cudaFree(d_kd);
      FDI_TRY(st);
    }
  }
  int* d_err = nullptr;
  FDI_TRY(dev_alloc(&d_err, 1));
  FDI_CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), s));
  fdi_status st = eigen_decompose_all(p->axes, s, d_err);
  if (st == FDI_OK) st = check_eigen_flag(d_err);
  cudaFree(d_err);
  FDI_TRY(st);
  FDI_TRY(finish_plan(p, s));
  if (p->prec != FDI_PREC_FP64) {
    std::vector<float> wyf(nr);
    std::vector<float2> wdf(nr);
    for (int i = 0; i < nr; ++i) {
      const double w = A[i] * g[i];
      wyf[i] = (float)w;
      const double v = g[i] / (h * h);
      const float vh = (float)v;
      wdf[i] = make_float2(vh, (float)(v - (double)vh));
    }
    FDI_TRY(upload(&p->cyl_wy_f, wyf));
    FDI_TRY(upload(&p->cyl_wres_df, wdf));
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

fdi_status fdi_plan_create_cyl(const double* rfaces, int nr, int ntheta, const double* zfaces, int nz,
                               fdi_bc bc_r_in, fdi_bc bc_r_out, fdi_bc bc_z_lo, fdi_bc bc_z_hi, fdi_precision prec,
                               int tpf, fdi_plan** out) {
  if (!out) return FDI_ERR_INVALID_ARG;
  *out = nullptr;
  if (!rfaces || !zfaces) return FDI_ERR_INVALID_ARG;
  if (nr < 2 || nr > kMaxN || nz < 2 || nz > kMaxN || ntheta < 3 || ntheta > kMaxN) {
    set_error("a cylindrical plan needs 2 <= n_r, n_z <= 256 and 3 <= n_theta <= 256 cells");
    return FDI_ERR_INVALID_ARG;
  }
  if (!(rfaces[0] >= 0.0)) {
    set_error("radial faces must be non-negative (rfaces[0] = 0 places the axis)");
    return FDI_ERR_INVALID_ARG;
  }
  for (int i = 0; i < nr; ++i)
    if (!(rfaces[i + 1] > rfaces[i]) || !std::isfinite(rfaces[i + 1])) {
      set_error("radial faces must be finite and strictly ascending");
      return FDI_ERR_INVALID_ARG;
    }
  for (int i = 0; i < nz; ++i)
    if (!(zfaces[i + 1] > zfaces[i]) || !std::isfinite(zfaces[i]) || !std::isfinite(zfaces[i + 1])) {
      set_error("axial faces must be finite and strictly ascending");
      return FDI_ERR_INVALID_ARG;
    }
  for (fdi_bc b : {bc_r_in, bc_r_out, bc_z_lo, bc_z_hi})
    if ((unsigned)b > 1u) return FDI_ERR_INVALID_ARG;
  if (tpf != 0 && tpf != 1) return FDI_ERR_INVALID_ARG;
  if (prec != FDI_PREC_FP64 && prec != FDI_PREC_MIXED_F16) {
    set_error("a cylindrical plan takes FDI_PREC_FP64 or FDI_PREC_MIXED_F16");
    return (prec == FDI_PREC_MIXED_TF32 || prec == FDI_PREC_MIXED_BF16) ? FDI_ERR_UNSUPPORTED : FDI_ERR_INVALID_ARG;
  }
  if (tpf && prec != FDI_PREC_FP64) {
    set_error("the cylindrical TPF (Eq. 45-46) runs on the FP64 path only");
    return FDI_ERR_UNSUPPORTED;
  }
  fdi_plan* p = new fdi_plan();
  p->grid = FDI_GRID_CELL;
  p->prec = prec;
  p->cyl = true;
  // external [z][theta][r] (r fastest) <-> internal [r][theta][z]: the x <-> z
  // swap of a Thomas-along-x plan
  p->thomas_ext = 0;
  p->perm[0] = 2;
  p->perm[2] = 0;
  p->thomas_axis = tpf ? -1 : 2;
  p->n[0] = nz;
  p->n[1] = ntheta;
  p->n[2] = nr;
  p->n_ext[0] = nr;
  p->n_ext[1] = ntheta;
  p->n_ext[2] = nz;
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
  fdi_status st = build_cyl_plan(p, rfaces, nr, ntheta, zfaces, nz, bc_r_in, bc_r_out, bc_z_lo, bc_z_hi, s);
  if (st == FDI_OK) {
    const size_t P = (size_t)nr * ntheta * nz;
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
