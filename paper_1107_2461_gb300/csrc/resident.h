// Resident small-grid solve: every pass of one or several mixed-precision
// field solves (TPT, Sec. 3, with the refinement rounds) in one cooperative
// launch.  Descriptor of one solve, built on the host from a plan's current
// workspace and passed to the kernel by value.
#pragma once
#include <cuda_runtime.h>

#include "fdi_internal.h"

namespace fdi {

constexpr int kResMaxJobs = 64;     // solves per launch
constexpr int kResMaxPlane = 128;   // largest x and y extent of a resident field

struct ResJob {
  int nx, ny, nz, px;      // extents; px: row pitch of the r and spectral planes (multiple of 4)
  int cls;                 // 64 or 128: padded extent of the plane products
  int singular;            // zero-flux Laplace problem (sigma = 0, zero-flux walls)
  int single_pass;         // one direct solve, FP64 output, no residual
  int vec;                 // residual pairs by vector accesses (nx even, FP64 arrays 16-byte aligned)
  int max_refine;
  int rgx, rgy, rgz, zchunk;  // residual grid of this shape
  int lt;                  // Thomas lines per unit (set at launch from the shared-memory size)
  double sigma, lambda, tol, fast_limit;
  const double* b;
  double* out;
  // transforms [forward E^{-1}, back E][axis x, y]: split-fp16 images in the
  // MMA's shared-memory layout (K chunks of 32, N_pad = 32 * k rows) and the
  // per-output power-of-two scales to undo; k = chunks of the axis
  int kx, ky;
  const uint8_t* img[2][2];
  const float* csc[2][2];
  // Thomas direction (z): eigenvalues of x and y, M, K diagonal and upper
  // off-diagonal of the z operator
  const double* lamx;
  const double* lamy;
  const float* mz;
  const float* kdz;
  const float* koz;
  // residual: double-float flux weights (unscaled) per direction [p, m, 0],
  // control-volume widths, and the lambda-scaled weights written per solve
  const float2* w[3][3];
  const float2* m[3];
  float2* lam_w;
  // workspace of the solve
  float* r;                // residual planes [z][y][x] (pitch px)
  float* F;                // spectral planes [z][j][i] (pitch px)
  float* cs;               // Thomas c' scratch (layout of F)
  float* xh;               // solution planes H, L, low part of L (P floats each)
  float* r1;               // r_1: hi planes, lo planes at r1 + r1_plane
  long long r1_plane;
  double* partials;
  DevStatus* st;
  unsigned* ticket;        // per-solve reduction ticket (zero between launches)
  float* rmax;             // scratch for the residual's max |r| (unused by this path)
};

// true when field `field` of plan p runs as a resident solve
bool resident_eligible(const fdi_plan* p, int field);
// descriptor of one solve on the plan's current workspace
fdi_status resident_describe(fdi_plan* p, int field, double sigma, double lambda, const double* rhs, double* out,
                             ResJob* job);
// one cooperative launch over `n` solves (n <= kResMaxJobs, no workspace
// shared between them); `owner` holds the grid barrier and the wait limit
fdi_status resident_launch(fdi_plan* owner, const ResJob* jobs, int n, cudaStream_t s);

}  // namespace fdi
