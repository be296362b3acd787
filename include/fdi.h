/*
 * fdi.h -- fast direct inverses of Helmholtz, Laplace and Stokes operators on
 * stretched finite-volume grids, for one NVIDIA GB300 (sm_103a).
 *
 * Method (Vitoshkin & Gelfgat, arXiv:1107.2461):
 *   - Sec. 3, Eq. 23-29: the discrete Laplacian on an orthogonal grid is a
 *     Kronecker sum of 1D operators D = E Lambda E^{-1} (Eq. 24); the Helmholtz
 *     and Laplace inverses are (E_x(x)E_y(x)E_z) Lambda^{-1} (E_x^{-1}(x)...) f
 *     (TPF, Eq. 29), or the same with the Thomas algorithm in one direction (TPT,
 *     end of Sec. 3);
 *   - Sec. 2, Eq. 8-9: the Stokes operator is inverted in three steps, only the
 *     pressure matrix C = sum_c D_c H_c^{-1} G_c being inverted iteratively, by a
 *     Krylov method preconditioned with the inverse pressure Laplacian.
 *
 * Conventions
 *   - Grids: per direction d (0 = x, 1 = y, 2 = z) the caller gives n[d] cells
 *     and n[d]+1 strictly ascending face coordinates.  Cell-centred unknowns
 *     use the finite-volume second derivative with the wall value imposed at
 *     half a cell (Dirichlet) or a zero wall flux (Neumann).
 *   - Fields are FP64, contiguous, C order [n_z][n_y][n_x] (x fastest), in
 *     device memory owned by the caller.
 *   - Operator: A = sigma*I - lambda*Delta.  fdi_helmholtz_solve uses sigma = 1
 *     (the paper's H = Delta - I/dt of Eq. 1 multiplied by -dt, with viscosity
 *     1/Re so lambda = dt/Re); fdi_laplace_solve uses sigma = 0, lambda = 1
 *     (-Delta u = f).  The pure zero-flux Laplacian is singular (Eq. 28): f is
 *     projected to zero volume-weighted mean and the zero-mean u is returned.
 *   - Staggered (MAC) grid, FDI_GRID_MAC: u on the interior x-faces
 *     ((n_x-1)*n_y*n_z values), v on the interior y-faces (n_x*(n_y-1)*n_z),
 *     w on the interior z-faces (n_x*n_y*(n_z-1)), p at the cells; no-slip
 *     walls.  fdi_stokes_solve solves
 *         (I - lambda*Delta_c) u_c + dt*(G p)_c = f_c,  D u = 0,  lambda = dt/Re
 *     (Eq. 8 scaled by -dt) and returns p with zero volume-weighted mean.
 *
 * Asynchrony: every solve is enqueued on `stream`.  Numerical results
 * (iterations, refinement steps, relative residual) are read with
 * fdi_last_result after the caller synchronises the stream.
 * fdi_stokes_solve on a capturable (non-default) stream with timing off runs
 * its Krylov loop on the device (a WHILE node of a CUDA graph repeats the
 * iteration until a device-side convergence flag is set) and needs no host
 * round trip; on the legacy default stream, or with per-kernel timing on, it
 * reads the convergence flag back after every iteration and so synchronises
 * `stream`.
 *
 * Threading: a plan owns one workspace.  Using one plan from two host threads,
 * or on two streams at once, is a data race.
 *
 * Errors: argument errors are returned synchronously and leave the outputs
 * untouched.  A CUDA error is returned as FDI_ERR_CUDA.  No C++ exception
 * crosses this interface.
 */
#ifndef FDI_H
#define FDI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* fdi_stream_t; /* the same handle as cudaStream_t; NULL = legacy default stream */
typedef struct fdi_plan fdi_plan;         /* opaque; owns every device buffer it allocates */

typedef enum {
  FDI_OK = 0,
  FDI_ERR_INVALID_ARG = 1,
  FDI_ERR_OUT_OF_MEMORY = 2,
  FDI_ERR_CUDA = 3,
  FDI_ERR_NOT_CONVERGED = 4,
  FDI_ERR_TIMEOUT = 5,
  FDI_ERR_SINGULAR = 6,
  FDI_ERR_UNSUPPORTED = 7
} fdi_status;

typedef enum { FDI_BC_DIRICHLET = 0, FDI_BC_NEUMANN = 1 } fdi_bc;
typedef enum { FDI_GRID_CELL = 0, FDI_GRID_MAC = 1 } fdi_grid;

/* Arithmetic of the x/y eigenvector transforms (the dense contractions of
 * Eq. 25/29).  FDI_PREC_FP64: every step in FP64.  The mixed modes split each
 * operand into a high and a low part in a 16-bit (or TF32) tensor-core type,
 * form hi*hi + hi*lo + lo*hi with FP32 accumulation, keep the intermediate
 * fields in FP32, run the Thomas sweep in FP32, and recover FP64 accuracy by
 * iterative refinement against a residual evaluated in double-float (about 48
 * significant bits) arithmetic.  Only the split-fp16 form is built: at FP32
 * accumulation it converges like a TF32 split at twice the tensor rate. */
typedef enum {
  FDI_PREC_FP64 = 0,
  FDI_PREC_MIXED_TF32 = 1, /* reserved, not built: fdi_plan_create returns FDI_ERR_UNSUPPORTED */
  FDI_PREC_MIXED_BF16 = 2, /* reserved, not built: fdi_plan_create returns FDI_ERR_UNSUPPORTED */
  FDI_PREC_MIXED_F16 = 3   /* split fp16 (hi + lo), the built mixed mode */
} fdi_precision;

/* Fields of a plan.  FDI_FIELD_CELL is the cell-centred grid (for a MAC plan:
 * the pressure grid, zero-flux walls). */
typedef enum { FDI_FIELD_CELL = 0, FDI_FIELD_U = 1, FDI_FIELD_V = 2, FDI_FIELD_W = 3 } fdi_field;

/* Create a plan: builds the 1D operators from the face coordinates (Sec. 3,
 * Eq. 23) and computes their eigen decompositions D = E Lambda E^{-1} (Eq. 24)
 * in FP64 on the current CUDA device -- O(n^3) once per grid, Sec. 3 -- and
 * keeps E, E^{-1}, Lambda and the workspace resident.
 *   faces[d]   host pointer to n[d]+1 ascending doubles (copied; not retained)
 *   n[d]       cells per direction, 2 <= n[d] <= 256
 *   bc_lo/hi   wall type of each side of each direction (FDI_GRID_CELL only;
 *              ignored for FDI_GRID_MAC, whose walls are no-slip)
 *   thomas_axis 0, 1, 2: TPT with the Thomas sweeps along x, y or z; -2: along
 *              the direction with the most cells (the paper's choice, Sec. 3;
 *              ties go to z, then y); -1: eigen decomposition in all three
 *              directions (TPF).  A cell plan with the Thomas axis x or y works
 *              on a copy of each field with that axis outermost: every solve
 *              permutes the right-hand side in and the solution out (two FP64
 *              copies of the field, owned by the plan).  Staggered (MAC) plans
 *              take 2 or -1.  Other values: FDI_ERR_UNSUPPORTED.  fdi_plan_eigen
 *              and fdi_apply_transform take the caller's directions.
 * Synchronous.  On error *out is set to NULL. */
fdi_status fdi_plan_create(const double* const faces[3], const int n[3], const fdi_bc bc_lo[3],
                           const fdi_bc bc_hi[3], fdi_grid grid, fdi_precision prec, int thomas_axis,
                           fdi_plan** out);

/* Create a plan on a cylindrical grid (Sec. 6, Eq. 41-46): the Helmholtz /
 * Poisson operator sigma*I - lambda*(D_rr + (1/r^2) D_thth + D_zz) in finite
 * volumes, on cells (r_i, theta_j, z_k) of an annulus or a full cylinder.
 *   rfaces   host, nr+1 ascending radial faces, rfaces[0] >= 0; rfaces[0] = 0
 *            makes the inner face the axis (a face of zero area: no flux, and
 *            bc_r_in is ignored)
 *   ntheta   uniform cells on the full circle, periodic
 *   zfaces   host, nz+1 ascending axial faces
 *   bc_*     wall types of the inner / outer radius and the two ends
 *   tpf      0: TPT, eigen transforms along theta and z and the Thomas
 *            algorithm along r per pair of modes (Eq. 42-44); 1: TPF, one
 *            radial eigen decomposition per theta mode (Eq. 45) and a divide
 *            (Eq. 46), FP64 plans only (else FDI_ERR_UNSUPPORTED)
 * Finite-volume reading (the paper prints no stencil): annular cell areas
 * A_i = (rho_{i+1}^2 - rho_i^2)/2, radial flux through rho_{i+1} equal to
 * rho_{i+1} (u_{i+1} - u_i) / (c_{i+1} - c_i) with c_i the cell centres, a
 * Dirichlet wall at half a cell, and the 1/r^2 of Eq. 41 as
 * g_i = (rho_{i+1} - rho_i) / (c_i A_i) per radial cell.  The theta
 * eigenbasis is the discrete Fourier basis in closed form; the z and r ones
 * are computed on the GPU as for fdi_plan_create.
 * Fields are FP64, C order [nz][ntheta][nr] (r fastest).  Limits:
 * 2 <= nr, nz <= 256, 3 <= ntheta <= 256.  Solves: fdi_helmholtz_solve,
 * fdi_laplace_solve and fdi_field_solve (FDI_FIELD_CELL) and their host and
 * batched forms; the singular zero-flux Laplacian (axis or zero-flux inner
 * wall, zero-flux outer wall and ends, sigma = 0) returns
 * FDI_ERR_UNSUPPORTED.  fdi_plan_eigen takes d = 0 (r), 1 (theta), 2 (z).
 * prec: FDI_PREC_FP64 or FDI_PREC_MIXED_F16.  Synchronous; *out = NULL on
 * error. */
fdi_status fdi_plan_create_cyl(const double* rfaces, int nr, int ntheta, const double* zfaces, int nz,
                               fdi_bc bc_r_in, fdi_bc bc_r_out, fdi_bc bc_z_lo, fdi_bc bc_z_hi, fdi_precision prec,
                               int tpf, fdi_plan** out);

/* Release every device buffer of the plan (synchronises the device first). */
fdi_status fdi_plan_destroy(fdi_plan* plan);

/* Convergence controls.  tol: target relative residual ||f - A u||/||f|| of the
 * Helmholtz/Laplace solves (default 1e-11 for FP64, 1e-10 mixed); max_refine:
 * refinement steps after the first solve (default 2 FP64, 3 mixed);
 * krylov_tol / max_iters: relative residual and iteration cap of the
 * pressure-matrix Krylov solve (defaults 1e-11 / 200). */
fdi_status fdi_plan_set_tolerances(fdi_plan* plan, double tol, int max_refine, double krylov_tol,
                                   int max_iters);

/* (I - lambda*Delta) out = rhs on the plan's cell grid (Eq. 27 scaled), lambda >= 0.
 * rhs, out: device, n_x*n_y*n_z doubles; out may alias rhs. */
fdi_status fdi_helmholtz_solve(fdi_plan* plan, double lambda, const double* rhs, double* out,
                               fdi_stream_t stream);

/* -Delta out = rhs on the plan's cell grid (Eq. 23; Eq. 28 for zero-flux walls). */
fdi_status fdi_laplace_solve(fdi_plan* plan, const double* rhs, double* out, fdi_stream_t stream);

/* (sigma*I - lambda*Delta_field) out = rhs on any field of the plan (sigma in
 * {0, 1}, lambda > 0; sigma = 0 only on the cell field).  Sizes as listed above. */
fdi_status fdi_field_solve(fdi_plan* plan, fdi_field field, double sigma, double lambda,
                           const double* rhs, double* out, fdi_stream_t stream);

/* fdi_field_solve for count right-hand sides held in HOST memory (Sec. 3 direct
 * inverse with refinement, once per right-hand side).  h_rhs[i], h_out[i]:
 * host arrays of the field's size (C order, FP64); h_out[i] may equal
 * h_rhs[i]; page-locked memory (cudaHostAlloc / cudaHostRegister) lets the
 * copies overlap the solves, pageable memory works serialised.  The solves are
 * pipelined: the host-to-device copy of right-hand side i+1 and the
 * device-to-host copy of solution i-1 run on two plan-owned copy streams while
 * solve i runs on `stream` (the default stream is replaced by a plan-owned
 * one).  Device staging for two right-hand sides and two solutions (4 x the
 * field size in doubles) is allocated by the plan on first use and kept until
 * fdi_plan_destroy.  Blocking: returns once every solution is in host memory.
 * rel_residual: NULL or count doubles, each solve's final relative residual.
 * Returns FDI_OK when every solve met its tolerance, else the status of the
 * first that did not (the message names its index); fdi_last_result then
 * describes the last solve. */
fdi_status fdi_field_solve_host(fdi_plan* plan, fdi_field field, double sigma, double lambda,
                                const double* const* h_rhs, double* const* h_out, int count,
                                double* rel_residual, fdi_stream_t stream);

/* Semi-direct Stokes inverse on a FDI_GRID_MAC plan (Sec. 2, three steps after
 * Eq. 9).  f[c], u[c]: device velocity fields (sizes above); p: device pressure.
 * Outputs must not alias inputs. */
fdi_status fdi_stokes_solve(fdi_plan* plan, double dt, double Re, const double* const f[3],
                            double* const u[3], double* p, fdi_stream_t stream);

/* Krylov method of fdi_stokes_solve for the pressure system C q = D u_hat
 * (Sec. 2): 0 BiCGstab (van der Vorst; default), 1 BiCGstab(2) (Sleijpen &
 * Fokkema's BiCGstab(l) with l = 2, the paper's choice), both right-
 * preconditioned, or 2 conjugate gradients on -C q = -D u_hat in the
 * volume-weighted inner product sum(V x y), in which C is self-adjoint and -C
 * and the preconditioner's negative are positive definite on zero-mean
 * pressures (one C-product per iteration); FP64 scalars on the device.
 * fdi_last_result reports iterations: outer ones for BiCGstab(2) (four
 * C-products each), two C-products each for BiCGstab, one for CG.
 * Other values: FDI_ERR_INVALID_ARG. */
fdi_status fdi_plan_set_krylov(fdi_plan* plan, int method);

/* Preconditioner of the pressure-matrix Krylov solve: mode 0 is the paper's
 * inverse pressure Laplacian L_p^{-1} (Sec. 2, after Eq. 9); mode 1 (default)
 * adds the viscous term, L_p^{-1} - lambda*I (Cahouet & Chabard 1988), which is
 * the exact inverse of C when the discrete operators commute and reduces to
 * mode 0 as dt -> 0; with mode 0 the iteration stagnates at large dt/Re. */
fdi_status fdi_plan_set_stokes_preconditioner(fdi_plan* plan, int mode);

/* count independent Helmholtz solves (plans[i] may repeat only if the solves
 * are meant to run one after another on that plan's workspace). */
fdi_status fdi_helmholtz_solve_batched(fdi_plan* const* plans, const double* lambdas,
                                       const double* const* rhs, double* const* out, int count,
                                       fdi_stream_t stream);

/* Results of the last solve on this plan; call after synchronising its stream.
 * iters: Krylov iterations (Stokes) or 0; refine_steps: solves after the first;
 * rel_residual: final relative residual (Helmholtz/Laplace: of A u = f;
 * Stokes: of the pressure-matrix system).  Any pointer may be NULL. */
fdi_status fdi_last_result(const fdi_plan* plan, int* iters, int* refine_steps,
                           double* rel_residual);

/* Copy the plan's 1D eigen data for direction d of a field to host buffers:
 * lam (m doubles), E and Einv (m*m doubles, row-major), m = unknowns along d.
 * Any pointer may be NULL.  Synchronous. */
fdi_status fdi_plan_eigen(const fdi_plan* plan, fdi_field field, int d, double* lam, double* E,
                          double* Einv, int* m);

/* One split-precision tensor-core transform pass on its own, for testing the
 * dominant kernel: out[r][k] = sum_j T[k][j] in[r][j] for r < rows, with
 * T = E_d^{-1} (inverse != 0, the forward transform of Eq. 25) or E_d of
 * direction d of a field; m = unknowns along d.  in/out: device FP32, row r at
 * r * pitch, pitch = m rounded up to a multiple of 4; in and out must not
 * overlap.  Needs a FDI_PREC_MIXED_F16 plan.  Asynchronous on stream. */
fdi_status fdi_apply_transform(fdi_plan* plan, fdi_field field, int d, int inverse, const float* in, float* out,
                               long long rows, fdi_stream_t stream);

/* Allocation-free eigen decomposition of one 1D operator (the same kernel as
 * plan creation).  No counterpart in the paper: it exists for callers that may
 * not allocate device memory -- code that runs where cudaMalloc is forbidden or
 * would stall (an allocation-free real-time or serving loop, a runtime that owns
 * every device allocation) -- and that still need the eigenbasis of a new grid.
 * It calls no cudaMalloc, cudaFree or other allocating routine: the kernel's
 * scratch (the 1D operator, its job descriptor, its convergence flag) lives in a
 * file-scope device array of 3*256+16 doubles, present on every device that
 * loads the library until the process exits.
 *   faces       host, n+1 ascending doubles; face_kind 0: n cell unknowns with
 *               the walls bc_lo / bc_hi; face_kind 1: the n-1 interior-face
 *               unknowns of a staggered velocity component (no-slip walls:
 *               bc_lo and bc_hi must both be FDI_BC_DIRICHLET, anything else
 *               is rejected with FDI_ERR_INVALID_ARG)
 *   lam, E, Einv device outputs: m, m*m, m*m doubles (m unknowns, row-major
 *               as fdi_plan_eigen)
 *   converged   optional host pointer: if given, the call synchronises `stream`
 *               and stores 1 if the QL iteration converged, else 0
 * Limits: 2 <= n <= 256 (3 <= n for face_kind 1); larger n is rejected with
 * FDI_ERR_INVALID_ARG.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress).  Every call copies the operator from
 * pageable host memory (and, with `converged`, synchronises `stream`), so no
 * call may be made while `stream` is being captured into a CUDA graph: a
 * capturing stream is rejected with FDI_ERR_INVALID_ARG.  Every call shares the
 * one array and overwrites it (the flag is cleared per call): calls that
 * overlap on the GPU, on any stream, race. */
fdi_status fdi_eigen_noalloc(const double* faces, int n, int face_kind, fdi_bc bc_lo, fdi_bc bc_hi, double* lam,
                             double* E, double* Einv, int* converged, fdi_stream_t stream);

/* Bound on every wait inside the kernels of a mixed plan that wait: the
 * tensor-core transforms (a CTA's roles hand shared-memory stages to one
 * another through mbarriers) and the grid barrier of the resident solve (its
 * CTAs meet between passes), in SM clock cycles; 0 restores the default of
 * 4e9 cycles (about two seconds at 2 GHz).  A transform wait that runs out
 * stops every role of its CTA, lets the asynchronous copies and MMAs already
 * issued finish, frees its tensor memory and returns; a barrier wait that runs
 * out raises an abort flag on which every CTA of the launch returns at its
 * next barrier.  The plan then records the failure in a flag that stays set, so
 * fdi_last_result (and every later solve's result) reports FDI_ERR_TIMEOUT,
 * until the next call of this function clears it.  The solution of a solve
 * that timed out is undefined.  Synchronises the device (the flag is cleared
 * once nothing runs); drops the plan's captured graphs.  FP64 plans accept
 * the call and have no such waits.  cycles < 0: FDI_ERR_INVALID_ARG. */
fdi_status fdi_plan_set_wait_limit(fdi_plan* plan, long long cycles);

/* Resident solve of mixed plans (enable = 1; default 0): a field whose x
 * and y extents are at most 128 is solved by one cooperative launch that runs
 * every pass of the TPT solve (Sec. 3, end) and of its refinement rounds, the
 * CTAs meeting at a grid barrier between passes; a z-plane fits in shared
 * memory there and one CTA applies both plane transforms to it in FP32.  The
 * three velocity solves of a Stokes step (fdi_stokes_solve) and the small
 * grids of fdi_helmholtz_solve_batched share such launches (up to 64 solves
 * each), with results bitwise equal to the same solve launched alone.
 * Cylindrical plans, TPF plans and larger fields always run pass by pass.
 * Each pass of the resident launch takes about 10 us on a 64^3 field (a
 * chain of dependent steps per unit), so a lone solve costs about what the
 * pass-by-pass graph costs (0.12 ms at 64^3) in one launch instead of 28;
 * for larger planes and for several solves per launch it is slower.
 * enable = 0: every field pass by pass (tensor-core transforms, one launch
 * per pass).  Drops the plan's captured graphs.  FP64 plans accept the call
 * and ignore it.  Other values: FDI_ERR_INVALID_ARG. */
fdi_status fdi_plan_set_resident(fdi_plan* plan, int enable);

/* Thomas sweep of mixed plans: 64 or 128 lines (one per thread) per CTA;
 * 2: two adjacent lines per thread, 64 threads per CTA (default); 3: as 2,
 * with the forward sweep's intermediate values of the top 128 planes kept in
 * shared memory instead of the field (64 KB per CTA).  These four are FP32
 * recurrences and a tuning knob: their results are bitwise identical.
 * 4: an FP64 recurrence on the FP32 fields with the line factors (reciprocal
 * pivots and c') cached per (sigma, lambda, field) in every workspace
 * (allocated by this call: 16 bytes per point per workspace); results differ
 * from the FP32 sweeps by rounding, within the refinement.  The singular
 * zero-flux Laplacian keeps the FP32 sweep.  FP64 plans always sweep in FP64
 * with such a cache.  Other values: FDI_ERR_INVALID_ARG. */
fdi_status fdi_plan_set_thomas_config(fdi_plan* plan, int lines_per_cta);

/* Autotuner for mixed plans: times `reps` complete Helmholtz solves
 * (sigma = 1, `lambda`, rhs -> out on `stream`, after one warm-up solve each)
 * for every Thomas configuration (2, 3, 64, 128), keeps the fastest on the plan
 * and records it for the plan's grid shape:
 * plans created later with the same shape and precision start with it.  Every
 * configuration computes bitwise-identical results.  rhs and out: device FP64
 * fields of the plan's cell shape, distinct; out is overwritten.  The chosen
 * value is written to *thomas_tl_out (host, may be NULL).
 * Synchronises `stream`.  FP64 plans have nothing to tune (returns OK). */
fdi_status fdi_plan_autotune(fdi_plan* plan, double lambda, const double* rhs, double* out, int reps,
                             int* thomas_tl_out, fdi_stream_t stream);

/* CUDA-graph replay of field solves (default on).  A Helmholtz / Laplace /
 * field solve whose arguments (field, sigma, lambda, rhs, out, stream) repeat
 * those of the previous call on this plan is captured into a CUDA graph on its
 * second occurrence and replayed as one graph launch from then on; results are
 * identical to the eager launch sequence.  The legacy default stream and plans
 * with timing on always run eagerly.  Changing tolerances or the Thomas
 * configuration drops the captured graph.  on: 0 off, nonzero on. */
fdi_status fdi_plan_set_graphs(fdi_plan* plan, int on);

/* Per-kernel device timing: with timing on, every kernel launch of this plan is
 * bracketed by a CUDA event pair on the launching stream. */
fdi_status fdi_plan_enable_timing(fdi_plan* plan, int on);

/* Harvest the recorded event pairs (synchronises on them) and report, per
 * kernel name, the accumulated device time in ms and the launch count since the
 * last reset.  names[i] stay valid until the plan is destroyed.  Up to `max`
 * entries are written; *count receives the number written. */
fdi_status fdi_plan_kernel_times(fdi_plan* plan, int max, const char** names, double* total_ms,
                                 long long* launches, int* count);

/* Harvest pending events and clear the accumulated kernel times. */
fdi_status fdi_plan_reset_kernel_times(fdi_plan* plan);

/* Number of kernels the last solve on this plan enqueued (host-side count). */
fdi_status fdi_last_launch_count(const fdi_plan* plan, long long* launches);

/* Human-readable text of the last error recorded on the calling host thread. */
const char* fdi_last_error_message(void);

const char* fdi_status_string(fdi_status s);

/* ---------------------------------------------------------------------------
 * Serving runtime (no counterpart in the paper, which applies the inverses
 * inside its own time stepper): a request loop for the Stokes-inverse
 * applications that time-stepper-based Newton and Arnoldi iterations issue
 * (Sec. 1-2), with uneven grids and differing dt / Re.  Plans and eigenbases
 * stay resident in a cache keyed by (n, beta, precision); requests are
 * admitted in FIFO order when their footprint (plan, if not cached, plus
 * fields) fits the device-memory budget, idle plans being evicted least
 * recently used; `slots` worker threads with one CUDA stream each run admitted
 * requests concurrently (continuous batching: a request arriving while others
 * run starts as soon as a slot and memory free up); requests of at most 128^3
 * cells run on high-priority streams, so the GPU dispatches their blocks ahead
 * of those of larger requests running at the same time.  Each request is solved
 * exactly as a lone fdi_stokes_solve on a plan of its grid, so its result does
 * not depend on the mix.
 * ------------------------------------------------------------------------- */
typedef struct fdi_server fdi_server;

/* One Stokes-inverse request on the no-slip unit box with n[d] cells per
 * direction (2 <= n[d] <= 256), faces x_i = (1 + tanh(beta (2i/n - 1)) /
 * tanh(beta)) / 2 in every direction (beta = 0: uniform), the staggered MAC
 * unknowns of fdi_stokes_solve, time step dt > 0, Reynolds number Re > 0,
 * precision FDI_PREC_FP64 or FDI_PREC_MIXED_F16.  f, u, p are HOST arrays in
 * the MAC shapes (u: (n_x-1) n_y n_z, v: n_x (n_y-1) n_z, w: n_x n_y (n_z-1),
 * p: n_x n_y n_z; x fastest), owned by the caller and left untouched (f) /
 * written (u, p) until the request is done. */
typedef struct {
  int n[3];
  double beta;
  double dt, Re;
  fdi_precision prec;
  const double* f[3];
  double* u[3];
  double* p;
} fdi_stokes_request;

typedef struct {
  int state;            /* 0 queued, 1 running, 2 done */
  fdi_status status;    /* of the solve (valid when done) */
  int iters;            /* BiCGstab iterations */
  double rel_residual;  /* relative residual of the pressure system */
  double queue_ms;      /* submission -> start */
  double latency_ms;    /* submission -> completion (when done) */
} fdi_stokes_result;

typedef struct {
  long long completed;
  double p50_ms, p99_ms;    /* latency percentiles over completed requests */
  double throughput_rps;    /* completed / (last completion - first submission) */
  size_t peak_bytes, bytes_in_use;
  long long plans_created, plans_evicted, plans_cached;
} fdi_server_report;

/* Device bytes a MAC Stokes plan of this size allocates (upper estimate used
 * for admission); prec: an fdi_precision value. */
size_t fdi_stokes_plan_bytes_estimate(const int n[3], int prec);

/* Start `slots` (1..64) workers on the current device with a device-memory
 * budget in bytes for plans plus request fields. */
fdi_status fdi_server_create(size_t hbm_budget_bytes, int slots, fdi_server** out);

/* Queue a request (returns at once).  FDI_ERR_OUT_OF_MEMORY if its footprint
 * alone exceeds the budget; FDI_ERR_INVALID_ARG / FDI_ERR_UNSUPPORTED for bad
 * fields.  *ticket identifies it. */
fdi_status fdi_server_submit(fdi_server* server, const fdi_stokes_request* req, long long* ticket);

/* State and result of a request; wait != 0 blocks until it is done. */
fdi_status fdi_server_poll(fdi_server* server, long long ticket, int wait, fdi_stokes_result* res);

/* Block until every submitted request is done. */
fdi_status fdi_server_drain(fdi_server* server);

/* Latency percentiles, throughput, memory and plan-cache counters. */
fdi_status fdi_server_stats(fdi_server* server, fdi_server_report* out);

/* Finish queued requests, stop the workers, free every cached plan. */
fdi_status fdi_server_destroy(fdi_server* server);

#ifdef __cplusplus
}
#endif

#endif /* FDI_H */
