// Internal declarations of libfdi: plan layout, device status, kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/fdi.h"

namespace fdi {

constexpr int kMaxN = 256;       // cells per direction supported by the plan
constexpr int kMaxRefineCap = 8;

// Device-side status of the last solve on a plan (written by kernels).
struct DevStatus {
  int done;          // refinement / Krylov converged: later rounds early-exit
  int refine_steps;  // solves after the first
  int iters;         // Krylov iterations
  int error;         // nonzero: numerical failure (non-finite residual ...)
  double rel_res;    // relative residual of the last check
  double bnorm2;     // ||b||^2 of the current solve
  double mean_b;     // volume-weighted mean of b (singular problems)
  double tol_used;   // tolerance the last solve was run to
  double scal[16];   // scratch scalars (volume-weighted mean of the solution, ...)
};

struct KryState;     // Krylov scalars of the Stokes pressure solve (stokes.cu)

// One 1D operator D = M^{-1} K along a direction (Eq. 23-24), resident on device.
struct Axis {
  int n = 0;
  bool zero_flux = false;           // both walls zero-flux: Lambda_0 = 0 exactly
  bool periodic = false;            // uniform periodic direction (cylindrical theta): closed-form eigenbasis
  // device arrays
  double* m = nullptr;              // M diagonal (control-volume widths), n
  double* kd = nullptr;             // K diagonal, n
  double* ko = nullptr;             // K off-diagonal K[i][i+1], n-1 (padded to n)
  double* wp = nullptr;             // flux weights K[i][i+1]/m_i, n (0 at the last index)
  double* wm = nullptr;             // K[i][i-1]/m_i, n (0 at index 0)
  double* w0 = nullptr;             // (K_ii + K_i,i+1 + K_i,i-1)/m_i: wall term, n
  double* lam = nullptr;            // eigenvalues, n, descending (closest to 0 first)
  double* E = nullptr;              // n*n row-major E[r][k]   (column k = eigenvector k)
  double* Einv = nullptr;           // n*n row-major Einv[k][r]
  // mixed-precision data of this operator (tensor-core matrices, FP32 and
  // double-float coefficients); owned, see mixed.cu
  void* mixed = nullptr;
  // host copies
  std::vector<double> h_m, h_kd, h_ko;
};

struct Field {
  Axis* ax[3] = {nullptr, nullptr, nullptr};
  int n[3] = {0, 0, 0};             // unknowns per direction
  long long P = 0;
  double vol_sum = 0.0;             // sum of control volumes
  bool zero_flux_all = false;       // singular when sigma = 0
};

}  // namespace fdi

// Per-solve device workspace of a plan.  A MAC plan owns three extra slots so
// that the u, v, w Helmholtz solves of a Stokes step can run concurrently.
struct fdi_work_slot {
  double* ws[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  float* wf[4] = {nullptr, nullptr, nullptr, nullptr};
  float2* xdf = nullptr;
  float* wr1 = nullptr;
  long long wr1_plane = 0;
  float* d_scales = nullptr;
  float2* lam_w = nullptr;
  double* partials = nullptr;
  fdi::DevStatus* d_status = nullptr;
  unsigned* d_counter = nullptr;
  double* tf = nullptr;             // Thomas factor cache (see fdi_plan::tf)
  long long tf_q = 0;
};

struct fdi_plan {
  fdi_grid grid;
  fdi_precision prec;
  int thomas_axis;                  // internal: 2 (TPT along the internal z) or -1 (TPF)
  // Thomas axis as the caller named it, and the external grid: a cell plan
  // whose Thomas axis is x or y works on a permuted copy of its fields
  // (internal axis d holds external axis perm[d]; see permute.cu)
  int thomas_ext = 2;
  int n_ext[3] = {0, 0, 0};
  int perm[3] = {0, 1, 2};
  double* tstage[2] = {nullptr, nullptr};  // right-hand side and solution in internal order
  int n[3];
  int device;
  std::vector<fdi::Axis*> axes;
  fdi::Field fields[4];
  int nfields = 1;
  long long Pmax = 0;
  // workspace (FP64 path): 5 buffers of Pmax doubles
  double* ws[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  // mixed-path workspace: FP32 buffers + double-float pairs
  float* wf[4] = {nullptr, nullptr, nullptr, nullptr};
  float2* xdf = nullptr;            // mixed solution planes H, L, low part of L (3 x Pmax floats)
  float* wr1 = nullptr;             // mixed: first residual r_1 as (hi, lo) FP32 planes
  long long wr1_plane = 0;
  float* d_scales = nullptr;        // per refinement round: max |field| of the pass inputs
  int* d_err = nullptr;             // nonzero: a kernel hit a wait limit (sticky)
  unsigned* res_bar = nullptr;      // grid barrier of the plan's resident launches (zero between launches)
  int resident = 0;                 // 1: mixed fields with x, y extents <= 128 solved by one resident launch
  long long wait_cycles = 0;        // bound of every tensor-core kernel wait, cycles (0: about 2 s)
  int thomas_tl = 2;                // FP32 Thomas: lines per CTA (64, 128) or 2 = two lines per thread
  float2* lam_w = nullptr;          // lambda-scaled double-float flux weights [3][3][kMaxN]
  unsigned* d_counter = nullptr;    // ticket counter of the fused last-block reductions (zero between launches)
  cudaStream_t cstream = nullptr;   // mixed plans: captures the bodies of conditional refinement rounds
  double* partials = nullptr;       // reduction partials
  int npartials = 0;
  // Thomas factor cache of this workspace: the reciprocal pivots and c' of
  // every z line ([k][line], tf_q doubles each) for the (sigma, lambda, field)
  // stored in the 4 doubles after them; a sweep whose arguments match reuses
  // them (decided on the device), any other sweep recomputes and stores them
  double* tf = nullptr;
  long long tf_q = 0;
  fdi::DevStatus* d_status = nullptr;
  int* h_flag = nullptr;            // pinned host flag for Krylov convergence
  // Stokes workspace (MAC plans): 10 cell vectors, 6 face fields, geometry
  double* sk[12] = {nullptr};
  double* skf[6] = {nullptr};
  double* mac_ih[3] = {nullptr, nullptr, nullptr};
  double* mac_idc[3] = {nullptr, nullptr, nullptr};
  fdi::KryState* d_kry = nullptr;
  fdi_work_slot extra[3];           // MAC plans: workspaces of the concurrent u, v, w solves
  int nextra = 0;
  cudaStream_t sstream[3] = {nullptr, nullptr, nullptr};  // streams of those solves
  cudaEvent_t sfork = nullptr, sjoin[3] = {nullptr, nullptr, nullptr};
  // cylindrical plans (Sec. 6, Eq. 41-46): internal x = z, y = theta
  // (periodic), z = r; the theta eigenvalue carries the radial factor g_i (the
  // discrete 1/r^2) in the Thomas sweep and in the residual
  bool cyl = false;
  double* cyl_wy = nullptr;         // FP64 [n_r]: A_i g_i, Thomas weight of the theta eigenvalue
  double* cyl_wres = nullptr;       // FP64 [n_r]: g_i / h_theta^2, theta flux weight of radial cell i
  float* cyl_wy_f = nullptr;        // FP32 copy of cyl_wy (mixed Thomas sweep)
  float2* cyl_wres_df = nullptr;    // double-float copy of cyl_wres (mixed residual)
  double* cyl_Er = nullptr;         // TPF: per theta mode j the radial E_{r,j} [n_theta][n_r][n_r] (Eq. 45)
  double* cyl_Eri = nullptr;        //      and E_{r,j}^{-1}
  double* cyl_lr = nullptr;         //      and its eigenvalues [n_theta][n_r]
  int stokes_precond = 1;           // 0: L_p^{-1} (paper), 1: L_p^{-1} - lambda I
  int krylov = 0;                   // 0: BiCGstab, 1: BiCGstab(2) (the paper's solver)
  double* kpartials = nullptr;
  unsigned* kticket = nullptr;      // last-block ticket of the Krylov reductions
  // controls
  double tol = 1e-11;
  int max_refine = 2;
  double ktol = 1e-11;
  int kmaxit = 200;
  // last results (host)
  int last_iters = 0, last_refine = 0;
  double last_res = 0.0;
  long long launches = 0;
  bool status_valid = false;
  // CUDA graphs of the field solve: a call that repeats the arguments (field,
  // sigma, lambda, arrays, stream) of one of the last few distinct calls is
  // captured on its second occurrence and replayed with a single graph launch
  // afterwards (a small LRU set, so alternating buffers keep their graphs)
  bool use_graphs = true;
  bool pdl = true;                  // programmatic dependent launch between the mixed solve's kernels
  // mixed field solves run one direct solve only (no residual check, no
  // refinement; FP64 output of the first solve): set around preconditioner
  // applications, which need no more than an approximate inverse
  bool single_pass = false;
  struct GraphKey {
    int field = -1;
    double sigma = 0.0, lambda = 0.0;
    const double* rhs = nullptr;
    double* out = nullptr;
    cudaStream_t s = nullptr;
  };
  static constexpr int kGraphSlots = 4;
  struct GraphSlot {
    GraphKey key;
    bool valid = false;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
    unsigned long long last_use = 0;
  };
  GraphSlot gslots[kGraphSlots];
  unsigned long long gclock = 0;
  // host-buffer solves (fdi_field_solve_host): device staging for two
  // right-hand sides and two solutions, copy streams and their events, and
  // the per-solve status records
  double* hstage[4] = {nullptr, nullptr, nullptr, nullptr};
  long long hstage_len = 0;
  cudaStream_t hcopy[3] = {nullptr, nullptr, nullptr};  // host-to-device, device-to-host, compute fallback
  cudaEvent_t hev[7] = {};          // in[2], solved[2], out[2], start
  fdi::DevStatus* d_hstat = nullptr;
  fdi::DevStatus* h_hstat = nullptr;  // pinned
  int hstat_cap = 0;
  // CUDA graph of one BiCGstab iteration of the Stokes inverse (every
  // iteration after the first enqueues the same launches on plan workspace)
  cudaGraphExec_t kgraph = nullptr;
  double kgraph_lambda = 0.0;
  int kgraph_precond = -1;
  int kgraph_krylov = -1;
  cudaStream_t kgraph_stream = nullptr;
  long long kgraph_launches = 0;
  long long kgraph_body_launches = 0;  // launches of one pass of the device-side Krylov loop
  long long kloop_body_launches = 0;   // the same for the last solve (0: no device-side loop)
  // optional per-kernel device timing (CUDA events around each launch)
  bool timing = false;
  struct TimedLaunch { const char* name; cudaEvent_t e0, e1; };
  std::vector<TimedLaunch> pending;
  std::vector<cudaEvent_t> event_pool;
  struct KernelTime { std::string name; double ms; long long n; };
  std::vector<KernelTime> ktimes;
};

namespace fdi {

// error helpers
void set_error(const std::string& msg);
fdi_status solve_status(const fdi_plan* plan, const DevStatus& st, int kerr);
void free_host_staging(fdi_plan* p);
long long stokes_loop_launches(const fdi_plan* p);
fdi_status launch_axis_permute(fdi_plan* p, const double* in, double* out, bool to_internal, cudaStream_t s);
#define FDI_CUDA_TRY(expr)                                                      \
  do {                                                                          \
    cudaError_t _e = (expr);                                                    \
    if (_e != cudaSuccess) {                                                    \
      ::fdi::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));     \
      return FDI_ERR_CUDA;                                                      \
    }                                                                           \
  } while (0)
#define FDI_LAUNCH_CHECK(plan)                                                  \
  do {                                                                          \
    (plan)->launches++;                                                         \
    cudaError_t _e = cudaGetLastError();                                        \
    if (_e != cudaSuccess) {                                                    \
      ::fdi::set_error(std::string("kernel launch: ") + cudaGetErrorString(_e)); \
      return FDI_ERR_CUDA;                                                      \
    }                                                                           \
  } while (0)

// Scoped per-kernel timer: records an event pair around the launches in its
// scope when timing is enabled on the plan.
struct KTimer {
  fdi_plan* p;
  const char* name;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr;
  KTimer(fdi_plan* p_, const char* name_, cudaStream_t s_);
  ~KTimer();
};
#define FDI_KTIMER(plan, name, stream) ::fdi::KTimer _kt_##__LINE__((plan), (name), (stream))

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization is launched while its predecessor in the stream completes and
// calls pdl_wait() before touching anything the predecessor writes (returns
// once the predecessor has completed and its memory is visible); a no-op for
// ordinary launches.  (Triggering the successor early measured slower, both
// as each CTA starts and, in the tensor-core transform, at each CTA's last
// tile: 0.641 against 0.597 ms per 256^3 solve.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// drop the captured solve graph (arguments or controls changed)
void invalidate_graph(fdi_plan* p);

// exchange the plan's per-solve workspace pointers with a slot (host side, so
// a solve enqueued in between uses the slot's buffers)
void swap_slot(fdi_plan* p, fdi_work_slot& w);
struct SlotSwap {
  fdi_plan* p;
  fdi_work_slot* w;
  SlotSwap(fdi_plan* p_, fdi_work_slot* w_) : p(p_), w(w_) {
    if (w) swap_slot(p, *w);
  }
  ~SlotSwap() {
    if (w) swap_slot(p, *w);
  }
};
// allocate / free the per-solve workspace held in the plan's own pointers
fdi_status alloc_workspace(fdi_plan* p);
void free_workspace(fdi_plan* p);
fdi_status mixed_alloc_workspace(fdi_plan* p);

// autotuned configurations per grid shape (fdi_plan_autotune records, plan
// creation applies)
void remember_tuning(const fdi_plan* p);
void apply_tuning(fdi_plan* p);

// independent Helmholtz solves of several plans: concurrent on a stream pool,
// one CUDA graph when the same batch repeats
fdi_status batch_solve(fdi_plan* const* plans, const double* lambdas, const double* const* rhs, double* const* out,
                       int count, cudaStream_t s);

// plan-time eigen decomposition of the symmetric tridiagonal M^{-1/2} K M^{-1/2}
// (periodic axes are skipped: their eigenbasis is set in closed form)
fdi_status eigen_decompose_all(const std::vector<Axis*>& axes, cudaStream_t s, int* d_err);
// `count` operators of size n sharing M and the off-diagonal of K, diagonal
// kd_all + q n for operator q; outputs at lam_all + q n, E_all / Einv_all + q n^2;
// operator 0 is given the exact null pair when zero_flux0
fdi_status eigen_decompose_batch(int count, int n, const double* m, const double* kd_all, const double* ko,
                                 bool zero_flux0, double* lam_all, double* E_all, double* Einv_all, cudaStream_t s,
                                 int* d_err);

// FP64 path launchers (kernels_f64.cu)
fdi_status launch_lines_f64(fdi_plan* p, const double* in, double* out, const double* T, int nin,
                            int nout, long long lines, bool accumulate, const int* skip, cudaStream_t s);
fdi_status launch_slab_f64(fdi_plan* p, const double* in, double* out, const double* T, int nin,
                           int nout, long long ncols, int batch, const int* skip, cudaStream_t s);
fdi_status launch_modes_f64(fdi_plan* p, const double* in, double* out, const double* T_all, int n, int nx,
                            int ny, const int* skip, cudaStream_t s);
fdi_status launch_divide_modes_f64(fdi_plan* p, const Field& f, double sigma, double lambda, double* data,
                                  const int* skip, cudaStream_t s);
// Thomas factor cache of the plan's current workspace: allocated for q line
// points (FP64 plans at creation, mixed plans when configuration 4 is chosen)
fdi_status alloc_thomas_cache(fdi_plan* p, long long q);
// cached-factor FP64 sweep over FP32 data in the mixed path's layout
// (configuration 4); f, layout and coefficients as the FP32 sweeps
fdi_status launch_thomas_cached_f32(fdi_plan* p, const Field& f, double sigma, double lambda, int field, float* data,
                                    int pitch, long long plane, float* fmax, const int* skip, cudaStream_t s);
fdi_status launch_thomas_f64(fdi_plan* p, const Field& f, double sigma, double lambda, int field, const double* in,
                             double* out, double* scratch, const int* skip, cudaStream_t s);
fdi_status launch_divide_f64(fdi_plan* p, const Field& f, double sigma, double lambda, double* data,
                             const int* skip, cudaStream_t s);
fdi_status launch_residual_f64(fdi_plan* p, const Field& f, double sigma, double lambda, const double* b,
                               const double* u, double* r, bool subtract_mean, const int* skip,
                               cudaStream_t s);
fdi_status launch_finish_residual(fdi_plan* p, int nblocks, bool first, int count_step, const int* skip,
                                  cudaStream_t s);
fdi_status launch_mean_f64(fdi_plan* p, const Field& f, const double* b, cudaStream_t s);
fdi_status launch_reset_status(fdi_plan* p, cudaStream_t s);

// solve orchestration (solve.cu)
fdi_status field_solve(fdi_plan* p, int field, double sigma, double lambda, const double* rhs, double* out,
                       cudaStream_t s);
fdi_status validate_field_args(const fdi_plan* p, int field, double sigma, double lambda);
fdi_status field_solve_entry(fdi_plan* p, int field, double sigma, double lambda, const double* rhs, double* out,
                             cudaStream_t s);

// mixed path (mixed.cu)
fdi_status mixed_setup(fdi_plan* p);
void mixed_free_axis(Axis* ax);

// Stokes (stokes.cu)
fdi_status stokes_setup(fdi_plan* p);
fdi_status stokes_solve(fdi_plan* p, double dt, double Re, const double* const f[3], double* const u[3], double* pr,
                        cudaStream_t s);
fdi_status mixed_field_solve(fdi_plan* p, int field, double sigma, double lambda, const double* rhs,
                             double* out, cudaStream_t s);

}  // namespace fdi
