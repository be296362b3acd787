// Semi-direct inverse of the staggered Stokes operator (Sec. 2).
//
// System (Eq. 8 scaled by -dt, viscosity 1/Re, lambda = dt/Re):
//     (I - lambda Delta_c) u_c + dt (G p)_c = f_c   (c = u, v, w),     D u = 0.
// Three steps (Sec. 2, after Eq. 9), with q = dt * p:
//   1. u_hat_c = H_c^{-1} f_c                                   (3 direct solves)
//   2. C q = D u_hat,  C = sum_c D_c H_c^{-1} G_c (Eq. 9), by BiCGstab preconditioned
//      with the inverse pressure Laplacian L_p^{-1}, L_p = D G (zero-flux, solved by
//      the same direct method); every C-product costs three direct Helmholtz solves
//   3. u_c = u_hat_c - H_c^{-1} (G q)_c                          (3 direct solves)
// Preconditioner: the paper's inverse pressure Laplacian L_p^{-1} (mode 0), or,
// by default (mode 1), L_p^{-1} - lambda I (Cahouet & Chabard, Int. J. Numer.
// Meth. Fluids 8, 1988): with H = I - lambda Delta and commuting discrete
// operators C = L_p (I - lambda L_p)^{-1}, whose inverse is exactly
// L_p^{-1} - lambda I; it reduces to the paper's choice as dt -> 0 and keeps
// the iteration count bounded at large dt, where L_p^{-1} alone stagnates.
// Krylov methods: BiCGstab (default), the paper's BiCGstab(2), or conjugate
// gradients in the volume-weighted inner product <x, y> = sum V x y, in which C
// is self-adjoint (D is minus the volume-weighted adjoint of G): -C and the
// preconditioners -L_p^{-1} and -L_p^{-1} + lambda I are positive definite on
// zero-mean pressures, and CG needs one C-product per iteration.
// The Krylov scalars, dot products and vector updates stay on the device in
// FP64 (deterministic two-stage reductions).  On a capturable stream the
// iterations after the first run as one CUDA graph whose WHILE node repeats a
// captured iteration until the device-side convergence flag is set (no host
// round trip per iteration); eagerly the host reads the flag after every
// iteration.  The pressure is returned with zero volume-weighted mean.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "fdi_internal.h"
#include "resident.h"

namespace fdi {

struct KryState {
  double rho, rho_old, alpha, omega;
  double bnorm2, rnorm2, rel;
  double tol;
  int iters, maxit, done, error;
  // BiCGstab(2): beta, the MGS coefficient tau_12, sigma_1, sigma_2 and the
  // polynomial coefficients gamma'_1, gamma'_2, gamma_1, gamma_2, gamma''_1
  double beta, tau12, sigma1, sigma2, gp1, gp2, g1, g2, gpp1;
  int loops;  // iterations run by the device-side loop of a captured solve
};

namespace {

constexpr int kDotBlocks = 152 * 4;
constexpr int kDotThreads = 256;

struct MacGeom {
  int nx, ny, nz;
  const double* ih[3];   // 1 / h_i (cell widths), n_d each
  const double* idc[3];  // 1 / (c_j - c_{j-1}), interior faces, n_d - 1 each
  const double* m[3];    // cell widths (volumes = products)
  const double* vol;     // cell volumes, [z][y][x]
};

// cell volumes m_x[i] m_y[j] m_z[k] of the pressure grid
__global__ void k_volumes(MacGeom g, double* __restrict__ vol) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(q % g.nx);
    const long long t = q / g.nx;
    const int j = (int)(t % g.ny), k = (int)(t / g.ny);
    vol[q] = g.m[0][i] * g.m[1][j] * g.m[2][k];
  }
}

// g_c = (G q)_c, or -(G q)_c with NEG, on the interior faces (Eq. 31's D_p):
// one FP64 difference and one product per face (GB300 runs FP64 at 2
// operations per clock per SM, so the sign is folded into the product)
template <bool NEG>
__global__ void k_grad(MacGeom g, const double* __restrict__ q, double* __restrict__ gu, double* __restrict__ gv,
                       double* __restrict__ gw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  if (i >= nx || j >= ny) return;
  const long long c = ((long long)k * ny + j) * nx + i;
  const double qc = q[c];
  const double sx = NEG ? -g.idc[0][min(i, nx - 2)] : g.idc[0][min(i, nx - 2)];
  const double sy = NEG ? -g.idc[1][min(j, ny - 2)] : g.idc[1][min(j, ny - 2)];
  const double sz = NEG ? -g.idc[2][min(k, nz - 2)] : g.idc[2][min(k, nz - 2)];
  if (i + 1 < nx) gu[((long long)k * ny + j) * (nx - 1) + i] = (q[c + 1] - qc) * sx;
  if (j + 1 < ny) gv[((long long)k * (ny - 1) + j) * nx + i] = (q[c + nx] - qc) * sy;
  if (k + 1 < nz) gw[((long long)k * ny + j) * nx + i] = (q[c + (long long)nx * ny] - qc) * sz;
}

// y = D h at the cells (Eq. 30's D_u), wall velocities zero
__global__ void k_div(MacGeom g, const double* __restrict__ hu, const double* __restrict__ hv,
                      const double* __restrict__ hw, double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  if (i >= nx || j >= ny) return;
  const long long ru = ((long long)k * ny + j) * (nx - 1);
  const double ur = (i + 1 < nx) ? hu[ru + i] : 0.0, ul = (i > 0) ? hu[ru + i - 1] : 0.0;
  const long long rv = (long long)k * (ny - 1) * nx;
  const double vr = (j + 1 < ny) ? hv[rv + (long long)j * nx + i] : 0.0;
  const double vl = (j > 0) ? hv[rv + (long long)(j - 1) * nx + i] : 0.0;
  const long long pw = (long long)ny * nx;
  const double wr = (k + 1 < nz) ? hw[(long long)k * pw + (long long)j * nx + i] : 0.0;
  const double wl = (k > 0) ? hw[(long long)(k - 1) * pw + (long long)j * nx + i] : 0.0;
  y[((long long)k * ny + j) * nx + i] = (ur - ul) * g.ih[0][i] + (vr - vl) * g.ih[1][j] + (wr - wl) * g.ih[2][k];
}

__device__ __forceinline__ void block_reduce2(double& a, double& b) {
  __shared__ double sh[2 * (kDotThreads / 32)];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x / 32, ln = threadIdx.x % 32;
  if (ln == 0) {
    sh[2 * w] = a;
    sh[2 * w + 1] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0, sb = 0;
    for (int q = 0; q < kDotThreads / 32; ++q) {
      sa += sh[2 * q];
      sb += sh[2 * q + 1];
    }
    a = sa;
    b = sb;
  }
}

__device__ void kry_finish_last(const double* partials, KryState* st, int kind, unsigned* ticket);

// partial sums of a.b and c.d (c, d may be null) over n values
__global__ void __launch_bounds__(kDotThreads) k_dot2(const double* __restrict__ a, const double* __restrict__ b,
                                                      const double* __restrict__ c, const double* __restrict__ d,
                                                      long long n, double* __restrict__ partials, KryState* fst, int fkind, unsigned* ticket) {
  double s0 = 0.0, s1 = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    s0 = fma(a[q], b[q], s0);
    if (c) s1 = fma(c[q], d[q], s1);
  }
  block_reduce2(s0, s1);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s0;
    partials[2 * blockIdx.x + 1] = s1;
  }
  kry_finish_last(partials, fst, fkind, ticket);
}

__device__ __forceinline__ void sum_partials(const double* partials, double& a, double& b) {
  a = 0.0;
  b = 0.0;
  for (int q = threadIdx.x; q < kDotBlocks; q += blockDim.x) {
    a += partials[2 * q];
    b += partials[2 * q + 1];
  }
  block_reduce2(a, b);
}

// kinds of scalar updates after a reduction (KF_L2_*: BiCGstab(2))
enum {
  KF_INIT = 0, KF_ALPHA = 1, KF_OMEGA = 2, KF_ITER = 3, KF_MEAN = 4,
  KF_L2_INIT = 5, KF_L2_RHO0 = 6, KF_L2_RHO = 7, KF_L2_ALPHA = 8, KF_L2_MR1 = 9, KF_L2_TAU = 10, KF_L2_MR2 = 11,
  KF_L2_CONV = 12, KF_CG_RHO = 13, KF_CG_ALPHA = 14, KF_CG_ITER = 15
};

// The scalar step after a reduction, by one block (every thread takes part
// in the fixed-order sum; thread 0 updates the state).
__device__ void kry_finish_body(const double* partials, KryState* st, int kind) {
  double a, b;
  sum_partials(partials, a, b);
  if (threadIdx.x != 0) return;
  if (st->done && kind != KF_INIT && kind != KF_MEAN) return;
  switch (kind) {
    case KF_INIT:  // a = ||b||^2 (= rhat.r)
      st->bnorm2 = a;
      st->rnorm2 = a;
      st->rho = a;
      st->rho_old = 1.0;
      st->alpha = 1.0;
      st->omega = 1.0;
      st->iters = 0;
      st->rel = a > 0.0 ? 1.0 : 0.0;
      st->done = a > 0.0 ? 0 : 1;
      st->error = 0;
      if (!isfinite(a)) {  // non-finite right-hand side
        st->error = 7;
        st->done = 1;
      }
      break;
    case KF_ALPHA:  // a = rhat.v
      if (a == 0.0 || !isfinite(a)) {
        st->error = 2;
        st->done = 1;
      } else {
        st->alpha = st->rho / a;
      }
      break;
    case KF_OMEGA:  // a = t.s, b = t.t
      if (b == 0.0 || !isfinite(b)) {
        st->omega = 0.0;
        st->error = st->error ? st->error : 3;
        st->done = 1;
      } else {
        st->omega = a / b;
      }
      break;
    case KF_ITER: {  // a = r.r, b = rhat.r
      st->iters += 1;
      st->rnorm2 = a;
      st->rho_old = st->rho;
      st->rho = b;
      const double rel = sqrt(a / st->bnorm2);
      st->rel = rel;
      if (!isfinite(rel)) {
        st->error = 4;
        st->done = 1;
      } else if (rel <= st->tol) {
        st->done = 1;
      } else if (st->iters >= st->maxit) {
        st->done = 1;
        st->error = 5;
      } else if (b == 0.0 || st->omega == 0.0) {
        st->done = 1;
        st->error = 6;
      }
      break;
    }
    case KF_MEAN:  // a = sum V x, b = sum V: store the mean in rho_old slot of a scratch state
      st->rnorm2 = a / b;
      break;
    // ---- BiCGstab(2) (Sleijpen & Fokkema), right-preconditioned, iterate y ----
    case KF_L2_INIT:  // a = ||b||^2; rho0 = 1, alpha = 0, omega = 1
      st->bnorm2 = a;
      st->rnorm2 = a;
      st->rho = 1.0;
      st->alpha = 0.0;
      st->omega = 1.0;
      st->iters = 0;
      st->rel = a > 0.0 ? 1.0 : 0.0;
      st->done = a > 0.0 ? 0 : 1;
      st->error = 0;
      if (!isfinite(a)) {  // non-finite right-hand side
        st->error = 7;
        st->done = 1;
      }
      break;
    case KF_L2_RHO0:  // new outer iteration: rho0 = -omega rho0, then the j = 0 step (a = rhat.r_0)
      st->rho = -st->omega * st->rho;
      // fall through
    case KF_L2_RHO: {  // a = rhat.r_j: beta = alpha rho1 / rho0, rho0 = rho1
      if (st->rho == 0.0 || !isfinite(a)) {
        st->error = 6;
        st->done = 1;
        break;
      }
      st->beta = st->alpha * a / st->rho;
      st->rho = a;
      break;
    }
    case KF_L2_ALPHA:  // a = rhat.u_{j+1}
      if (a == 0.0 || !isfinite(a)) {
        st->error = 2;
        st->done = 1;
      } else {
        st->alpha = st->rho / a;
      }
      break;
    case KF_L2_MR1:  // a = r_1.r_1, b = r_0.r_1
      if (a == 0.0 || !isfinite(a)) {
        st->error = 3;
        st->done = 1;
      } else {
        st->sigma1 = a;
        st->gp1 = b / a;
      }
      break;
    case KF_L2_TAU:  // a = r_2.r_1
      st->tau12 = a / st->sigma1;
      break;
    case KF_L2_MR2:  // a = r_2.r_2 (after orthogonalisation), b = r_0.r_2
      if (a == 0.0 || !isfinite(a)) {
        st->error = 3;
        st->done = 1;
      } else {
        st->sigma2 = a;
        st->gp2 = b / a;
        st->g2 = st->gp2;
        st->omega = st->g2;
        st->g1 = st->gp1 - st->tau12 * st->g2;
        st->gpp1 = st->g2;
      }
      break;
    // ---- conjugate gradients (volume-weighted inner product) ----
    case KF_CG_RHO: {  // a = <r, z>, b = <v, z> (v = A p of the last step):
      // Polak-Ribiere beta = <r - r_old, z> / rho_old = -alpha b / rho_old
      if (!(a > 0.0) || !isfinite(a)) {
        st->error = 2;
        st->done = 1;
        break;
      }
      st->beta = st->iters > 0 ? -st->alpha * b / st->rho : 0.0;
      st->rho = a;
      break;
    }
    case KF_CG_ALPHA:  // a = <p, A p>
      if (!(a > 0.0) || !isfinite(a)) {
        st->error = 2;
        st->done = 1;
      } else {
        st->alpha = st->rho / a;
      }
      break;
    case KF_CG_ITER: {  // a = r.r after the update
      st->iters += 1;
      st->rnorm2 = a;
      const double rel = sqrt(a / st->bnorm2);
      st->rel = rel;
      if (!isfinite(rel)) {
        st->error = 4;
        st->done = 1;
      } else if (rel <= st->tol) {
        st->done = 1;
      } else if (st->iters >= st->maxit) {
        st->done = 1;
        st->error = 5;
      }
      break;
    }
    case KF_L2_CONV: {  // a = r_0.r_0 after the minimal-residual update
      st->iters += 1;
      st->rnorm2 = a;
      const double rel = sqrt(a / st->bnorm2);
      st->rel = rel;
      if (!isfinite(rel)) {
        st->error = 4;
        st->done = 1;
      } else if (rel <= st->tol) {
        st->done = 1;
      } else if (st->iters >= st->maxit) {
        st->done = 1;
        st->error = 5;
      } else if (st->omega == 0.0) {
        st->done = 1;
        st->error = 6;
      }
      break;
    }
  }
}

// The producing kernel's last block to finish (atomic ticket after its
// partials are visible) runs the scalar step and re-arms the ticket, so the
// reduction needs no second launch; the order of the sums is that of a
// separate finishing launch.
__device__ void kry_finish_last(const double* partials, KryState* st, int kind, unsigned* ticket) {
  __shared__ int last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1 ? 1 : 0;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  kry_finish_body(partials, st, kind);
  if (threadIdx.x == 0) *ticket = 0u;
}

// ---- BiCGstab(2) vector updates (all read the device scalars) ----

// j = 0: u_0 = r_0 - beta u_0;  j = 1: also u_1 = r_1 - beta u_1
__global__ void k_l2_u(const KryState* __restrict__ st, double* __restrict__ u0, double* __restrict__ u1,
                       const double* __restrict__ r0, const double* __restrict__ r1, long long n, int j) {
  if (st->done) return;
  const double be = st->beta;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    u0[q] = r0[q] - be * u0[q];
    if (j) u1[q] = r1[q] - be * u1[q];
  }
}

// j = 0: r_0 -= alpha u_1, y += alpha u_0;  j = 1: also r_1 -= alpha u_2
__global__ void k_l2_r(const KryState* __restrict__ st, double* __restrict__ r0, double* __restrict__ r1,
                       const double* __restrict__ u0, const double* __restrict__ u1, const double* __restrict__ u2,
                       double* __restrict__ y, long long n, int j) {
  if (st->done) return;
  const double al = st->alpha;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    r0[q] -= al * u1[q];
    if (j) r1[q] -= al * u2[q];
    y[q] += al * u0[q];
  }
}

// r_2 -= tau_12 r_1 (modified Gram-Schmidt)
__global__ void k_l2_tau(const KryState* __restrict__ st, double* __restrict__ r2, const double* __restrict__ r1,
                         long long n) {
  if (st->done) return;
  const double t = st->tau12;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    r2[q] -= t * r1[q];
}

// minimal-residual update: y += g1 r_0 + g''1 r_1, r_0 -= g'2 r_2 + g'1 r_1,
// u_0 -= g2 u_2 + g1 u_1; partial sums of r_0.r_0
__global__ void __launch_bounds__(kDotThreads) k_l2_final(const KryState* st, double* __restrict__ y,
                                                          double* __restrict__ r0, const double* __restrict__ r1,
                                                          const double* __restrict__ r2, double* __restrict__ u0,
                                                          const double* __restrict__ u1,
                                                          const double* __restrict__ u2, long long n,
                                                          double* __restrict__ partials, KryState* fst, int fkind, unsigned* ticket) {
  const bool live = !st->done;
  const double g1 = st->g1, g2 = st->g2, gp1 = st->gp1, gp2 = st->gp2, gpp1 = st->gpp1;
  double s0 = 0.0, s1 = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    if (live) {
      const double r0q = r0[q], r1q = r1[q];
      y[q] += g1 * r0q + gpp1 * r1q;
      const double rn = r0q - gp2 * r2[q] - gp1 * r1q;
      r0[q] = rn;
      u0[q] -= g2 * u2[q] + g1 * u1[q];
      s0 = fma(rn, rn, s0);
    }
  }
  block_reduce2(s0, s1);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s0;
    partials[2 * blockIdx.x + 1] = s1;
  }
  kry_finish_last(partials, fst, fkind, ticket);
}

// x = -t
__global__ void k_neg(double* __restrict__ x, const double* __restrict__ t, long long n) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    x[q] = -t[q];
}

// x = -x
__global__ void k_negate(double* __restrict__ x, long long n) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    x[q] = -x[q];
}

// p = r + beta (p - omega v),  beta = (rho / rho_old)(alpha / omega)
__global__ void k_bicg_p(const KryState* __restrict__ st, double* __restrict__ p, const double* __restrict__ r,
                         const double* __restrict__ v, long long n, int first) {
  if (st->done) return;
  const double beta = first ? 0.0 : (st->rho / st->rho_old) * (st->alpha / st->omega);
  const double om = st->omega;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    p[q] = first ? r[q] : r[q] + beta * (p[q] - om * v[q]);
}

// s = r - alpha v
__global__ void k_bicg_s(const KryState* __restrict__ st, double* __restrict__ s, const double* __restrict__ r,
                         const double* __restrict__ v, long long n) {
  if (st->done) return;
  const double al = st->alpha;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    s[q] = r[q] - al * v[q];
}

// x <- x + alpha phat + omega shat with phat = -y, shat = -z (the Laplace solves
// return -L_p^{-1}); r = s - omega t; partial sums of r.r and rhat.r
__global__ void __launch_bounds__(kDotThreads) k_bicg_xr(const KryState* st, double* __restrict__ x,
                                                         const double* __restrict__ y, const double* __restrict__ z,
                                                         double* __restrict__ r, const double* __restrict__ s,
                                                         const double* __restrict__ t,
                                                         const double* __restrict__ rhat, long long n,
                                                         double* __restrict__ partials, KryState* fst, int fkind, unsigned* ticket) {
  const bool live = !st->done;
  const double al = st->alpha, om = st->omega;
  double s0 = 0.0, s1 = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    if (live) {
      x[q] = x[q] - al * y[q] - om * z[q];
      const double rq = s[q] - om * t[q];
      r[q] = rq;
      s0 = fma(rq, rq, s0);
      s1 = fma(rhat[q], rq, s1);
    }
  }
  block_reduce2(s0, s1);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s0;
    partials[2 * blockIdx.x + 1] = s1;
  }
  kry_finish_last(partials, fst, fkind, ticket);
}

// partial sums of V x and V over the cells
__global__ void __launch_bounds__(kDotThreads) k_vsum(MacGeom g, const double* __restrict__ x,
                                                      double* __restrict__ partials, KryState* fst, int fkind, unsigned* ticket) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  double s0 = 0.0, s1 = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const double v = g.vol[q];
    s0 = fma(v, x[q], s0);
    s1 += v;
  }
  block_reduce2(s0, s1);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s0;
    partials[2 * blockIdx.x + 1] = s1;
  }
  kry_finish_last(partials, fst, fkind, ticket);
}

// p = (x - mean) / dt
__global__ void k_pressure(const KryState* __restrict__ mst, const double* __restrict__ x, double inv_dt,
                           double* __restrict__ p, long long n) {
  const double mu = mst->rnorm2;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    p[q] = (x[q] - mu) * inv_dt;
}

__global__ void k_sub(double* __restrict__ u, const double* __restrict__ h, long long n) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    u[q] -= h[q];
}

// y <- y + c x  (adds the viscous part of the pressure preconditioner)
__global__ void k_axpy(double* __restrict__ y, double c, const double* __restrict__ x, long long n) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    y[q] = fma(c, x[q], y[q]);
}

// ---- conjugate gradients ----

// partial sums of sum V a b and sum V c b (c may be null) over the cells
// (V = cell volume)
__global__ void __launch_bounds__(kDotThreads) k_wdot(MacGeom g, const double* __restrict__ a,
                                                      const double* __restrict__ b, const double* __restrict__ c,
                                                      double* __restrict__ partials, KryState* fst, int fkind, unsigned* ticket) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  double s0 = 0.0, s1 = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    const double vb = g.vol[q] * b[q];
    s0 = fma(vb, a[q], s0);
    if (c) s1 = fma(vb, c[q], s1);
  }
  block_reduce2(s0, s1);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s0;
    partials[2 * blockIdx.x + 1] = s1;
  }
  kry_finish_last(partials, fst, fkind, ticket);
}

// p = z (first iteration) or z + beta p
__global__ void k_cg_p(const KryState* __restrict__ st, double* __restrict__ p, const double* __restrict__ z,
                       long long n, int first) {
  if (st->done) return;
  const double be = st->beta;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    p[q] = first ? z[q] : fma(be, p[q], z[q]);
}

// x += alpha p, r -= alpha v (v = A p); partial sums of r.r
__global__ void __launch_bounds__(kDotThreads) k_cg_xr(const KryState* st, double* __restrict__ x,
                                                       double* __restrict__ r, const double* __restrict__ p,
                                                       const double* __restrict__ v, long long n,
                                                       double* __restrict__ partials, KryState* fst, int fkind, unsigned* ticket) {
  const bool live = !st->done;
  const double al = st->alpha;
  double s0 = 0.0, s1 = 0.0;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
    if (live) {
      x[q] = fma(al, p[q], x[q]);
      const double rq = fma(-al, v[q], r[q]);
      r[q] = rq;
      s0 = fma(rq, rq, s0);
    }
  }
  block_reduce2(s0, s1);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = s0;
    partials[2 * blockIdx.x + 1] = s1;
  }
  kry_finish_last(partials, fst, fkind, ticket);
}

__global__ void k_zero(double* __restrict__ a, long long n) {
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    a[q] = 0.0;
}

__global__ void k_stokes_report(const KryState* __restrict__ st, DevStatus* ds) {
  ds->iters = st->iters;
  ds->refine_steps = 0;
  ds->rel_res = st->rel;
  ds->error = st->error == 7 ? 7 : (st->error ? 1 : 0);
  ds->done = 1;
  ds->tol_used = st->tol;
}

__global__ void k_kry_setup(KryState* st, double tol, int maxit) {
  st->tol = tol;
  st->maxit = maxit;
  st->done = 0;
  st->error = 0;
  st->iters = 0;
  st->loops = 0;
}

// Device-side Krylov loop of a captured solve: a WHILE graph node runs one
// iteration per pass while its condition is set.  k_loop_init sets it before
// the node from the state after the first (eager) iteration; k_loop_cond, the
// last node of every pass, sets it again.  Every pass runs k_loop_cond, and
// the pass count is capped by the iteration limit independently of the done
// flag, so the loop ends after at most maxit passes.
__global__ void k_loop_init(KryState* st, cudaGraphConditionalHandle h) {
  st->loops = 0;
  cudaGraphSetConditional(h, (st->done == 0 && st->maxit > 1) ? 1u : 0u);
}

__global__ void k_loop_cond(KryState* st, cudaGraphConditionalHandle h) {
  st->loops += 1;
  cudaGraphSetConditional(h, (st->done == 0 && st->loops + 1 < st->maxit) ? 1u : 0u);
}

#define FDI_TRY(expr)            \
  do {                           \
    fdi_status _s = (expr);      \
    if (_s != FDI_OK) return _s; \
  } while (0)

template <typename T>
fdi_status dalloc(T** p, size_t n) {
  cudaError_t e = cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FDI_ERR_OUT_OF_MEMORY : FDI_ERR_CUDA;
  }
  return FDI_OK;
}

MacGeom geom(const fdi_plan* p) {
  MacGeom g;
  g.nx = p->n[0];
  g.ny = p->n[1];
  g.nz = p->n[2];
  for (int d = 0; d < 3; ++d) {
    g.ih[d] = p->mac_ih[d];
    g.idc[d] = p->mac_idc[d];
    g.m[d] = p->fields[FDI_FIELD_CELL].ax[d]->m;
  }
  g.vol = p->sk[10];
  return g;
}

}  // namespace

fdi_status stokes_setup(fdi_plan* p) {
  // geometry of the staggered derivatives, from the cell-Neumann operators' widths
  for (int d = 0; d < 3; ++d) {
    const std::vector<double>& h = p->fields[FDI_FIELD_CELL].ax[d]->h_m;
    const int n = (int)h.size();
    std::vector<double> ih(n), idc(std::max(1, n - 1));
    for (int i = 0; i < n; ++i) ih[i] = 1.0 / h[i];
    for (int j = 1; j < n; ++j) idc[j - 1] = 1.0 / (0.5 * (h[j - 1] + h[j]));
    FDI_TRY(dalloc(&p->mac_ih[d], n));
    FDI_TRY(dalloc(&p->mac_idc[d], idc.size()));
    FDI_CUDA_TRY(cudaMemcpy(p->mac_ih[d], ih.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    FDI_CUDA_TRY(cudaMemcpy(p->mac_idc[d], idc.data(), idc.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
  const long long Pc = p->fields[FDI_FIELD_CELL].P;
  long long Pf = 0;
  for (int c = 1; c <= 3; ++c) Pf = std::max(Pf, p->fields[c].P);
  for (int i = 0; i < 11; ++i) FDI_TRY(dalloc(&p->sk[i], Pc));   // b x r rhat p v s t y z, cell volumes
  for (int i = 0; i < 6; ++i) FDI_TRY(dalloc(&p->skf[i], Pf));  // g_u g_v g_w h_u h_v h_w
  {
    // on a private stream (plans may be created while other threads capture
    // or run work on theirs)
    cudaStream_t vs = nullptr;
    FDI_CUDA_TRY(cudaStreamCreateWithFlags(&vs, cudaStreamNonBlocking));
    const MacGeom g = geom(p);
    k_volumes<<<kDotBlocks, kDotThreads, 0, vs>>>(g, p->sk[10]);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(vs);
    cudaStreamDestroy(vs);
    FDI_CUDA_TRY(e);
  }
  FDI_TRY(dalloc(&p->d_kry, 2));
  FDI_TRY(dalloc(&p->kpartials, 2 * kDotBlocks));
  FDI_TRY(dalloc(&p->kticket, 1));
  FDI_CUDA_TRY(cudaMemset(p->kticket, 0, sizeof(unsigned)));
  return FDI_OK;
}

namespace {

// H_c^{-1} in_c -> out_c for c = u, v, w: the three solves run concurrently on
// the plan's side streams, each with its own workspace slot, forked from and
// joined back to s (also inside a stream capture)
fdi_status three_solves(fdi_plan* p, double lambda, const double* const in[3], double* const out[3],
                        cudaStream_t s) {
  if (p->nextra >= 3 && p->tstage[0] == nullptr && resident_eligible(p, 1) && resident_eligible(p, 2) &&
      resident_eligible(p, 3)) {
    // small grids: the three solves share one resident launch (every pass of
    // all three, each on its own workspace slot)
    ResJob jobs[3];
    for (int c = 0; c < 3; ++c) {
      SlotSwap guard(p, &p->extra[c]);
      FDI_TRY(resident_describe(p, 1 + c, 1.0, lambda, in[c], out[c], &jobs[c]));
    }
    FDI_KTIMER(p, "resident", s);
    return resident_launch(p, jobs, 3, s);
  }
  if (p->nextra < 3) {
    for (int c = 0; c < 3; ++c) FDI_TRY(field_solve(p, 1 + c, 1.0, lambda, in[c], out[c], s));
    return FDI_OK;
  }
  FDI_CUDA_TRY(cudaEventRecord(p->sfork, s));
  for (int c = 0; c < 3; ++c) {
    FDI_CUDA_TRY(cudaStreamWaitEvent(p->sstream[c], p->sfork, 0));
    {
      SlotSwap guard(p, &p->extra[c]);
      FDI_TRY(field_solve(p, 1 + c, 1.0, lambda, in[c], out[c], p->sstream[c]));
    }
    FDI_CUDA_TRY(cudaEventRecord(p->sjoin[c], p->sstream[c]));
    FDI_CUDA_TRY(cudaStreamWaitEvent(s, p->sjoin[c], 0));
  }
  return FDI_OK;
}

fdi_status cmatvec(fdi_plan* p, const MacGeom& g, double lambda, double* q, double* out, cudaStream_t s) {
  // out = C (-q) = -sum_c D_c H_c^{-1} G_c q   (q holds -phat, see k_bicg_xr)
  dim3 blk(32, 8), grd((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
  {
    FDI_KTIMER(p, "stokes_grad", s);
    k_grad<true><<<grd, blk, 0, s>>>(g, q, p->skf[0], p->skf[1], p->skf[2]);
    FDI_LAUNCH_CHECK(p);
  }
  {
    const double* in[3] = {p->skf[0], p->skf[1], p->skf[2]};
    double* out3[3] = {p->skf[3], p->skf[4], p->skf[5]};
    FDI_TRY(three_solves(p, lambda, in, out3, s));
  }
  FDI_KTIMER(p, "stokes_div", s);
  k_div<<<grd, blk, 0, s>>>(g, p->skf[3], p->skf[4], p->skf[5], out);
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

fdi_status wdots(fdi_plan* p, const MacGeom& g, const double* a, const double* b, const double* c, int kind,
                 cudaStream_t s) {
  FDI_KTIMER(p, "stokes_dot", s);
  k_wdot<<<kDotBlocks, kDotThreads, 0, s>>>(g, a, b, c, p->kpartials, p->d_kry, kind, p->kticket);
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

fdi_status dots(fdi_plan* p, const double* a, const double* b, const double* c, const double* d, long long n,
                int kind, cudaStream_t s) {
  FDI_KTIMER(p, "stokes_dot", s);
  k_dot2<<<kDotBlocks, kDotThreads, 0, s>>>(a, b, c, d, n, p->kpartials, p->d_kry, kind, p->kticket);
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

}  // namespace

fdi_status stokes_solve(fdi_plan* p, double dt, double Re, const double* const f[3], double* const u[3], double* pr,
                        cudaStream_t s) {
  const double lambda = dt / Re;
  const MacGeom g = geom(p);
  const long long Pc = p->fields[FDI_FIELD_CELL].P;
  double *b = p->sk[0], *x = p->sk[1], *r = p->sk[2], *rhat = p->sk[3], *pv = p->sk[4], *v = p->sk[5];
  double *sv = p->sk[6], *t = p->sk[7], *y = p->sk[8], *z = p->sk[9];
  const unsigned vb = 152 * 4, vt = 256;
  const dim3 blk(32, 8), grd((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
  // step 1: predictors u_hat_c = H_c^{-1} f_c, kept in the outputs
  FDI_TRY(three_solves(p, lambda, f, u, s));
  // b = D u_hat; r = rhat = b; x = p = v = 0
  k_div<<<grd, blk, 0, s>>>(g, u[0], u[1], u[2], b);
  FDI_LAUNCH_CHECK(p);
  k_kry_setup<<<1, 1, 0, s>>>(p->d_kry, p->ktol, p->kmaxit);
  FDI_LAUNCH_CHECK(p);
  FDI_CUDA_TRY(cudaMemcpyAsync(r, b, Pc * sizeof(double), cudaMemcpyDeviceToDevice, s));
  FDI_CUDA_TRY(cudaMemcpyAsync(rhat, b, Pc * sizeof(double), cudaMemcpyDeviceToDevice, s));
  k_zero<<<vb, vt, 0, s>>>(x, Pc);
  FDI_LAUNCH_CHECK(p);
  // step 2: Krylov solve of C q = b, right-preconditioned by L_p^{-1} (or its
  // Cahouet-Chabard form).  Iterations after the first replay one captured
  // graph of the iteration (plan workspace only, so the launches are
  // identical); the legacy stream and timed plans run eagerly.
  const bool graphs = p->use_graphs && !p->timing && s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
  auto run_loop = [&](auto&& iteration) -> fdi_status {
    p->kloop_body_launches = 0;
    if (!graphs) {
      // eager: one iteration at a time, the host reads the convergence flag
      for (int it = 0; it < p->kmaxit; ++it) {
        FDI_TRY(iteration(it == 0 ? 1 : 0));
        FDI_CUDA_TRY(cudaMemcpyAsync(p->h_flag, &p->d_kry->done, sizeof(int), cudaMemcpyDeviceToHost, s));
        FDI_CUDA_TRY(cudaStreamSynchronize(s));
        if (*p->h_flag) break;
      }
      return FDI_OK;
    }
    // the first iteration eagerly, the rest as one graph: a WHILE node whose
    // body is one iteration, so the loop runs on the device without a host
    // round trip per iteration
    FDI_TRY(iteration(1));
    if (!p->kgraph || p->kgraph_lambda != lambda || p->kgraph_precond != p->stokes_precond ||
        p->kgraph_krylov != p->krylov || p->kgraph_stream != s) {
      if (p->kgraph) cudaGraphExecDestroy(p->kgraph);
      p->kgraph = nullptr;
      const long long before = p->launches;
      cudaGraph_t gr = nullptr, body = nullptr;
      cudaGraphConditionalHandle h = 0;
      fdi_status st = FDI_OK;
      FDI_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaGraph_t g = nullptr;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd);
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault);
        if (e == cudaSuccess) {
          k_loop_init<<<1, 1, 0, s>>>(p->d_kry, h);
          e = cudaGetLastError();
          p->launches++;
        }
        if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd);
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t node = nullptr;
        if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp);
        if (e == cudaSuccess)
          e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
        if (e == cudaSuccess) {
          body = cp.conditional.phGraph_out[0];
        } else {
          set_error(std::string("Krylov loop node: ") + cudaGetErrorString(e));
          st = FDI_ERR_CUDA;
        }
      }
      cudaError_t e = cudaStreamEndCapture(s, &gr);
      if (st != FDI_OK || e != cudaSuccess || gr == nullptr) {
        if (gr) cudaGraphDestroy(gr);
        cudaGetLastError();
        if (st != FDI_OK) return st;
        FDI_CUDA_TRY(e);
        set_error("stream capture of the Krylov loop failed");
        return FDI_ERR_CUDA;
      }
      // the loop body: one iteration, then the loop condition
      const long long body_start = p->launches;
      e = cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        st = iteration(0);
        if (st == FDI_OK) {
          k_loop_cond<<<1, 1, 0, s>>>(p->d_kry, h);
          p->launches++;
          if (cudaGetLastError() != cudaSuccess) st = FDI_ERR_CUDA;
        }
        cudaGraph_t bg = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(s, &bg);
        if (st == FDI_OK && e2 != cudaSuccess) {
          set_error(std::string("stream capture of the Krylov iteration: ") + cudaGetErrorString(e2));
          st = FDI_ERR_CUDA;
        }
      } else {
        set_error(std::string("stream capture of the Krylov iteration: ") + cudaGetErrorString(e));
        st = FDI_ERR_CUDA;
      }
      const long long body_launches = p->launches - body_start;
      cudaGraphExec_t ex = nullptr;
      if (st == FDI_OK) {
        e = cudaGraphInstantiate(&ex, gr, 0);
        if (e != cudaSuccess) {
          set_error(std::string("Krylov loop graph: ") + cudaGetErrorString(e));
          st = FDI_ERR_CUDA;
        }
      }
      cudaGraphDestroy(gr);
      if (st != FDI_OK) {
        cudaGetLastError();
        return st;
      }
      p->kgraph = ex;
      p->kgraph_lambda = lambda;
      p->kgraph_precond = p->stokes_precond;
      p->kgraph_krylov = p->krylov;
      p->kgraph_stream = s;
      p->kgraph_launches = p->launches - before;
      p->kgraph_body_launches = body_launches;
      p->launches = before;
    }
    FDI_CUDA_TRY(cudaGraphLaunch(p->kgraph, s));
    // the loop init launch; the body's launches are counted once the number of
    // passes is known (fdi_last_launch_count)
    p->launches += p->kgraph_launches - p->kgraph_body_launches;
    p->kloop_body_launches = p->kgraph_body_launches;
    return FDI_OK;
  };
  // -(M^{-1} v) into `out`: the Laplace solve returns -L_p^{-1} v; mode 1 adds lambda v
  // The preconditioner only has to approximate C^{-1}: for CG and BiCGstab a
  // mixed plan applies its Laplace inverse as one direct solve without
  // refinement (CG takes the Polak-Ribiere coefficient, which tolerates the
  // slightly varying operator; BiCGstab builds the solution from the
  // preconditioned directions themselves).  BiCGstab(2) recovers q by one more
  // application at the end and keeps the refined solve.
  const bool approx_precond = p->prec != FDI_PREC_FP64 && p->krylov != 1;
  auto precond = [&](const double* vin, double* vout) -> fdi_status {
    p->single_pass = approx_precond;
    const fdi_status pst = field_solve(p, FDI_FIELD_CELL, 0.0, 1.0, vin, vout, s);
    p->single_pass = false;
    FDI_TRY(pst);
    if (p->stokes_precond == 1) {
      k_axpy<<<vb, vt, 0, s>>>(vout, lambda, vin, Pc);
      FDI_LAUNCH_CHECK(p);
    }
    return FDI_OK;
  };
  if (p->krylov == 2) {
    // conjugate gradients on (-C) y = b (y = -q) in the volume-weighted inner
    // product, preconditioned by precond() = -L_p^{-1} (+ lambda I); x = y, r,
    // z = preconditioned residual, pv = search direction, v = -C pv
    FDI_TRY(dots(p, b, b, nullptr, nullptr, Pc, KF_INIT, s));
    auto iteration = [&](int first) -> fdi_status {
      FDI_TRY(precond(r, z));
      FDI_TRY(wdots(p, g, r, z, first ? nullptr : v, KF_CG_RHO, s));
      k_cg_p<<<vb, vt, 0, s>>>(p->d_kry, pv, z, Pc, first);
      FDI_LAUNCH_CHECK(p);
      FDI_TRY(cmatvec(p, g, lambda, pv, v, s));
      FDI_TRY(wdots(p, g, pv, v, nullptr, KF_CG_ALPHA, s));
      {
        FDI_KTIMER(p, "stokes_update", s);
        k_cg_xr<<<kDotBlocks, kDotThreads, 0, s>>>(p->d_kry, x, r, pv, v, Pc, p->kpartials, p->d_kry, KF_CG_ITER,
                                                   p->kticket);
        FDI_LAUNCH_CHECK(p);
      }
      return FDI_OK;
    };
    FDI_TRY(run_loop(iteration));
    k_negate<<<vb, vt, 0, s>>>(x, Pc);  // q = -y
    FDI_LAUNCH_CHECK(p);
  } else if (p->krylov == 1) {
    // BiCGstab(2) (Sleijpen & Fokkema; the paper's solver, Sec. 2) on
    // (C M^{-1}) y = b; q = M^{-1} y at the end.  Vectors: x = y, r = r_0,
    // pv = u_0, v = u_1, sv = u_2, t = r_1, y = r_2, z = work.
    double *r0 = r, *u0 = pv, *u1 = v, *u2 = sv, *r1 = t, *r2 = y, *w = z;
    k_zero<<<vb, vt, 0, s>>>(u0, Pc);
    FDI_LAUNCH_CHECK(p);
    FDI_TRY(dots(p, b, b, nullptr, nullptr, Pc, KF_L2_INIT, s));
    auto op = [&](const double* vin, double* vout) -> fdi_status {  // vout = C M^{-1} vin
      FDI_TRY(precond(vin, w));
      return cmatvec(p, g, lambda, w, vout, s);
    };
    auto iteration = [&](int) -> fdi_status {
      // BiCG step j = 0
      FDI_TRY(dots(p, rhat, r0, nullptr, nullptr, Pc, KF_L2_RHO0, s));
      k_l2_u<<<vb, vt, 0, s>>>(p->d_kry, u0, u1, r0, r1, Pc, 0);
      FDI_LAUNCH_CHECK(p);
      FDI_TRY(op(u0, u1));
      FDI_TRY(dots(p, rhat, u1, nullptr, nullptr, Pc, KF_L2_ALPHA, s));
      k_l2_r<<<vb, vt, 0, s>>>(p->d_kry, r0, r1, u0, u1, u2, x, Pc, 0);
      FDI_LAUNCH_CHECK(p);
      FDI_TRY(op(r0, r1));
      // BiCG step j = 1
      FDI_TRY(dots(p, rhat, r1, nullptr, nullptr, Pc, KF_L2_RHO, s));
      k_l2_u<<<vb, vt, 0, s>>>(p->d_kry, u0, u1, r0, r1, Pc, 1);
      FDI_LAUNCH_CHECK(p);
      FDI_TRY(op(u1, u2));
      FDI_TRY(dots(p, rhat, u2, nullptr, nullptr, Pc, KF_L2_ALPHA, s));
      k_l2_r<<<vb, vt, 0, s>>>(p->d_kry, r0, r1, u0, u1, u2, x, Pc, 1);
      FDI_LAUNCH_CHECK(p);
      FDI_TRY(op(r1, r2));
      // minimal-residual step over r_0, r_1, r_2
      FDI_TRY(dots(p, r1, r1, r0, r1, Pc, KF_L2_MR1, s));
      FDI_TRY(dots(p, r2, r1, nullptr, nullptr, Pc, KF_L2_TAU, s));
      k_l2_tau<<<vb, vt, 0, s>>>(p->d_kry, r2, r1, Pc);
      FDI_LAUNCH_CHECK(p);
      FDI_TRY(dots(p, r2, r2, r0, r2, Pc, KF_L2_MR2, s));
      {
        FDI_KTIMER(p, "stokes_update", s);
        k_l2_final<<<kDotBlocks, kDotThreads, 0, s>>>(p->d_kry, x, r0, r1, r2, u0, u1, u2, Pc, p->kpartials,
                                                      p->d_kry, KF_L2_CONV, p->kticket);
        FDI_LAUNCH_CHECK(p);
      }
      return FDI_OK;
    };
    FDI_TRY(run_loop(iteration));
    // q = M^{-1} y
    FDI_TRY(precond(x, w));
    k_neg<<<vb, vt, 0, s>>>(x, w, Pc);
    FDI_LAUNCH_CHECK(p);
  } else {
    FDI_TRY(dots(p, b, b, nullptr, nullptr, Pc, KF_INIT, s));
    auto iteration = [&](int first) -> fdi_status {
      k_bicg_p<<<vb, vt, 0, s>>>(p->d_kry, pv, r, v, Pc, first);
      FDI_LAUNCH_CHECK(p);
      // y = (-L_p)^{-1} p (+ lambda p) = -phat ; v = C phat
      FDI_TRY(precond(pv, y));
      FDI_TRY(cmatvec(p, g, lambda, y, v, s));
      FDI_TRY(dots(p, rhat, v, nullptr, nullptr, Pc, KF_ALPHA, s));
      k_bicg_s<<<vb, vt, 0, s>>>(p->d_kry, sv, r, v, Pc);
      FDI_LAUNCH_CHECK(p);
      FDI_TRY(precond(sv, z));
      FDI_TRY(cmatvec(p, g, lambda, z, t, s));
      FDI_TRY(dots(p, t, sv, t, t, Pc, KF_OMEGA, s));
      {
        FDI_KTIMER(p, "stokes_update", s);
        k_bicg_xr<<<kDotBlocks, kDotThreads, 0, s>>>(p->d_kry, x, y, z, r, sv, t, rhat, Pc, p->kpartials, p->d_kry,
                                                     KF_ITER, p->kticket);
        FDI_LAUNCH_CHECK(p);
      }
      return FDI_OK;
    };
    FDI_TRY(run_loop(iteration));
  }
  // zero-mean pressure q -> p = q / dt
  {
    k_vsum<<<kDotBlocks, kDotThreads, 0, s>>>(g, x, p->kpartials, p->d_kry + 1, KF_MEAN, p->kticket);
    FDI_LAUNCH_CHECK(p);
    k_pressure<<<vb, vt, 0, s>>>(p->d_kry + 1, x, 1.0 / dt, pr, Pc);
    FDI_LAUNCH_CHECK(p);
  }
  // step 3: u_c = u_hat_c - H_c^{-1} (G q)_c   (x holds q; grad with +1)
  k_grad<false><<<grd, blk, 0, s>>>(g, x, p->skf[0], p->skf[1], p->skf[2]);
  FDI_LAUNCH_CHECK(p);
  {
    const double* in[3] = {p->skf[0], p->skf[1], p->skf[2]};
    double* out3[3] = {p->skf[3], p->skf[4], p->skf[5]};
    FDI_TRY(three_solves(p, lambda, in, out3, s));
  }
  for (int c = 0; c < 3; ++c) {
    k_sub<<<vb, vt, 0, s>>>(u[c], p->skf[3 + c], p->fields[1 + c].P);
    FDI_LAUNCH_CHECK(p);
  }
  k_stokes_report<<<1, 1, 0, s>>>(p->d_kry, p->d_status);
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

// launches run by the device-side Krylov loop of the last Stokes solve (its
// pass count is read from the device)
long long stokes_loop_launches(const fdi_plan* p) {
  if (!p || p->kloop_body_launches == 0 || !p->d_kry) return 0;
  int loops = 0;
  if (cudaMemcpy(&loops, &p->d_kry->loops, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return 0;
  return (long long)loops * p->kloop_body_launches;
}

}  // namespace fdi

using namespace fdi;

extern "C" fdi_status fdi_stokes_solve(fdi_plan* plan, double dt, double Re, const double* const f[3],
                                       double* const u[3], double* p, fdi_stream_t stream) {
  if (!plan || !f || !u || !p) return FDI_ERR_INVALID_ARG;
  if (plan->grid != FDI_GRID_MAC) {
    set_error("fdi_stokes_solve needs a FDI_GRID_MAC plan");
    return FDI_ERR_INVALID_ARG;
  }
  if (!(dt > 0.0) || !(Re > 0.0) || !std::isfinite(dt) || !std::isfinite(Re)) {
    set_error("dt and Re must be finite and positive");
    return FDI_ERR_INVALID_ARG;
  }
  for (int c = 0; c < 3; ++c)
    if (!f[c] || !u[c]) return FDI_ERR_INVALID_ARG;
  plan->launches = 0;
  plan->kloop_body_launches = 0;
  return stokes_solve(plan, dt, Re, f, u, p, (cudaStream_t)stream);
}

extern "C" fdi_status fdi_plan_set_krylov(fdi_plan* plan, int method) {
  if (!plan || method < 0 || method > 2) return FDI_ERR_INVALID_ARG;
  plan->krylov = method;
  return FDI_OK;
}

extern "C" fdi_status fdi_plan_set_stokes_preconditioner(fdi_plan* plan, int mode) {
  if (!plan || (mode != 0 && mode != 1)) return FDI_ERR_INVALID_ARG;
  plan->stokes_precond = mode;
  return FDI_OK;
}
