// FP64 kernels of the direct Helmholtz / Laplace inverse (the plain FP64 path).
//
//   k_lines_f64   out[l][k] = sum_j T[k][j] in[l][j]     transform along x (Eq. 25/29,
//                 the factor E_x^{-1} or E_x applied to every x-line)
//   k_slab_f64    out[b][k][c] = sum_j T[k][j] in[b][j][c]  transform along y per
//                 z-slab, or along z over all columns (TPF)
//   k_thomas_f64  per (x-mode, y-mode) line the tridiagonal z-system
//                 [(sigma - lam (Lx_i + Ly_j)) M_z - lam K_z] u = M_z f   (TPT,
//                 end of Sec. 3: Thomas algorithm in one direction)
//   k_divide_f64  u_ijk = f_ijk / (sigma - lam (Lx_i + Ly_j + Lz_k))  (Eq. 26-28)
//   k_residual_f64 r = b - A u with the 7-point finite-volume stencil in flux form,
//                 and per-block partial sums of r^2 and b^2 (fixed grid, so the
//                 reduction order is deterministic)
//
// GB300 runs FP64 at about 2 FMA/clk/SM, so the transforms are FP64-pipe bound;
// they are register-tiled (4x4 outputs per thread, 64x64 tiles staged in shared
// memory) so that every shared-memory load feeds two FMAs.
#include <cmath>

#include "fdi_internal.h"

namespace fdi {
namespace {

constexpr int TB = 64;   // tile edge
constexpr int TK = 16;   // k-chunk
constexpr int kResBlocks = 152 * 8;
constexpr int kResThreads = 256;

template <bool ACC>
__global__ void __launch_bounds__(256) k_lines_f64(const double* __restrict__ A, double* __restrict__ C,
                                                   const double* __restrict__ T, int nin, int nout,
                                                   long long L, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double As[TK][TB + 1];  // [j][line]
  __shared__ double Bs[TK][TB + 1];  // [j][k]
  const long long l0 = (long long)blockIdx.x * TB;
  const int k0 = blockIdx.y * TB;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int j0 = 0; j0 < nin; j0 += TK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int jj = threadIdx.x % TK, ll = threadIdx.x / TK + 16 * r;
      long long line = l0 + ll;
      int j = j0 + jj, k = k0 + ll;
      As[jj][ll] = (line < L && j < nin) ? A[line * nin + j] : 0.0;
      Bs[jj][ll] = (k < nout && j < nin) ? T[(long long)k * nin + j] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < TK; ++jj) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[jj][ty + 16 * q];
        b[q] = Bs[jj][tx + 16 * q];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[q][c] = fma(a[q], b[c], acc[q][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    long long line = l0 + ty + 16 * q;
    if (line >= L) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int k = k0 + tx + 16 * c;
      if (k < nout) {
        long long idx = line * nout + k;
        C[idx] = ACC ? C[idx] + acc[q][c] : acc[q][c];
      }
    }
  }
}

// Element (j, c) of the input of batch b at A[b * zin + j * rs + c], of the
// output C[b * zout + k * rs + c]; the matrix of batch b is T + b * tz (tz = 0:
// one matrix for every batch).  A y pass over z-slabs has rs = ncols, zin =
// nin * ncols; a per-mode transform (cylindrical TPF: one radial matrix per
// theta mode) has batch = mode, rs = the row stride of the field, tz = nin * nout.
__global__ void __launch_bounds__(256) k_slab_f64(const double* __restrict__ A, double* __restrict__ C,
                                                  const double* __restrict__ T, int nin, int nout,
                                                  long long ncols, long long rs, long long zin, long long zout,
                                                  long long tz, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double As[TK][TB + 1];  // T tile [j][k]
  __shared__ double Bs[TK][TB + 1];  // data tile [j][c]
  const long long b = blockIdx.z;
  A += b * zin;
  C += b * zout;
  T += b * tz;
  const long long c0 = (long long)blockIdx.x * TB;
  const int k0 = blockIdx.y * TB;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[a][q] = 0.0;
  for (int j0 = 0; j0 < nin; j0 += TK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int jj = threadIdx.x % TK, kk = threadIdx.x / TK + 16 * r;
      int j = j0 + jj, k = k0 + kk;
      As[jj][kk] = (k < nout && j < nin) ? T[(long long)k * nin + j] : 0.0;
      int cc = threadIdx.x % TB, jr = threadIdx.x / TB + 4 * r;
      long long col = c0 + cc;
      int j2 = j0 + jr;
      Bs[jr][cc] = (col < ncols && j2 < nin) ? A[(long long)j2 * rs + col] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < TK; ++jj) {
      double a[4], bb[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = As[jj][ty + 16 * q];
        bb[q] = Bs[jj][tx + 16 * q];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[q][c] = fma(a[q], bb[c], acc[q][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    int k = k0 + ty + 16 * q;
    if (k >= nout) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      long long col = c0 + tx + 16 * c;
      if (col < ncols) C[(long long)k * rs + col] = acc[q][c];
    }
  }
}

// Thomas sweep along z (TPT, end of Sec. 3) in FP64 for every (x-mode,
// y-mode) line: [(sigma - lam Lx_i) M_z - lam K_z - lam Ly_j W] u = M_z f with
// W = M_z (Cartesian) or the theta weight A g (cylindrical plans).  The line
// factorisation (c'_k and the reciprocal pivots) depends on (sigma, lambda,
// field) only; it is kept in a per-workspace cache whose key the sweep reads
// on the device: a matching key runs the cached sweep (about four FP64
// operations per point, no divide), any other runs the factorising sweep and
// refreshes the cache (the key is written by a one-thread kernel after it, so
// every block of a sweep sees the same key, also in replayed graphs).  T is
// the field type: double (FP64 path) or float (the mixed path's FP32 fields,
// configuration 4, FP64 recurrence).  Field element (k, line l) at
// k * kstride + (l / ny) * pitch + l % ny, l = i * ny + j ... for the FP64
// path pitch = ny = lines per x mode is replaced by the [z][y][x] order below.
struct ThomasArgs {
  const void* in;
  void* out;
  double* cs;        // scratch c'_k (no cache)
  int nx, ny, nz;
  int mixed_layout;  // 0: FP64 field [z][y][x] (line l = j*nx + i); 1: FP32 [z][i][pitch] (l = i*ny + j)
  int pitch;
  long long kstride;
  const double* lamx;
  const double* lamy;
  const double* mz;
  const double* kdz;
  const double* koz;
  const double* wy;  // per z: weight of the y eigenvalue (cylindrical theta: A_i g_i); null: M_z
  double sigma, lambda;
  int field;
  int singular_possible;  // sigma == 0 and zero-flux walls everywhere
  double* cinv;      // factor cache: reciprocal pivots [k][line] (null: no cache)
  double* ccp;       //               c'_k [k][line]
  const double* key; //               (sigma, lambda, field) of the cached factors
  long long q;       // line points per plane of the cache (>= lines)
  float* fmax;       // FP32 fields: atomic max |u| (the next pass's scale)
};

__device__ __forceinline__ void warp_max_out(float v, float* fmax) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v > 0.f) atomicMax(reinterpret_cast<unsigned int*>(fmax), __float_as_uint(v));
}

template <typename T>
__global__ void __launch_bounds__(128) k_thomas_f64(ThomasArgs a, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double s_m[kMaxN], s_lo[kMaxN];  // M_k and lambda K_{k,k+1}
  const int nz = a.nz;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    s_m[k] = a.mz[k];
    s_lo[k] = a.lambda * a.koz[k];
  }
  __syncthreads();
  const long long NL = (long long)a.nx * a.ny;
  const long long l0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float vmax = 0.f;
  // lines past the end run line NL - 1 again without storing (the warp stays
  // whole for the max reduction)
  const bool live = l0 < NL;
  const long long l = live ? l0 : NL - 1;
  int i, j;
  long long off;
  if (a.mixed_layout) {
    i = (int)(l / a.ny);
    j = (int)(l % a.ny);
    off = (long long)i * a.pitch + j;
  } else {
    i = (int)(l % a.nx);
    j = (int)(l / a.nx);
    off = l;
  }
  const T* in = static_cast<const T*>(a.in) + off;
  T* out = static_cast<T*>(a.out) + off;
  const long long ks = a.kstride;
  const double lab = a.lamx[i] + a.lamy[j];
  // the y eigenvalue takes its own weight on cylindrical plans (Eq. 44: the
  // theta eigenvalue multiplies the discrete 1/r^2 of the radial cell)
  const double s = a.sigma - a.lambda * (a.wy ? a.lamx[i] : lab);
  const double ly = a.wy ? a.lambda * a.lamy[j] : 0.0;
  const double lam = a.lambda;
  if (!(a.singular_possible && lab == 0.0)) {
    const bool cached = a.cinv && a.key[0] == a.sigma && a.key[1] == a.lambda && a.key[2] == (double)a.field;
    double* cp_arr = a.cinv ? a.ccp + l : a.cs + off;
    const long long cstride = a.cinv ? a.q : ks;
    if (cached && live) {
      const double* inv = a.cinv + l;
      double d = 0.0;
      for (int k = 0; k < nz; ++k) {
        double t = __dmul_rn(s_m[k], (double)in[k * ks]);
        if (k > 0) t = __fma_rn(s_lo[k - 1], d, t);
        d = __dmul_rn(t, inv[k * a.q]);
        out[k * ks] = (T)d;
      }
      double u = d;
      vmax = fmaxf(vmax, fabsf((float)u));
      for (int k = nz - 2; k >= 0; --k) {
        u = __fma_rn(-cp_arr[k * cstride], u, (double)out[k * ks]);
        out[k * ks] = (T)u;
        vmax = fmaxf(vmax, fabsf((float)u));
      }
    } else if (live) {
      double cprev = 0.0, dprev = 0.0;
      for (int k = 0; k < nz; ++k) {
        const double lo = (k > 0) ? -s_lo[k - 1] : 0.0;
        const double up = (k + 1 < nz) ? -s_lo[k] : 0.0;
        double di = s * s_m[k] - lam * a.kdz[k];
        if (a.wy) di -= ly * a.wy[k];
        const double inv = 1.0 / (di - lo * cprev);
        cprev = up * inv;
        // the same operations, in the same order, as the cached sweep: a
        // solve gives the same bits whether its factors were cached or not
        double t = __dmul_rn(s_m[k], (double)in[k * ks]);
        if (k > 0) t = __fma_rn(s_lo[k - 1], dprev, t);
        dprev = __dmul_rn(t, inv);
        cp_arr[k * cstride] = cprev;
        if (a.cinv) a.cinv[l + k * a.q] = inv;
        out[k * ks] = (T)dprev;
      }
      double u = dprev;
      vmax = fmaxf(vmax, fabsf((float)u));
      for (int k = nz - 2; k >= 0; --k) {
        u = __fma_rn(-cp_arr[k * cstride], u, (double)out[k * ks]);
        out[k * ks] = (T)u;
        vmax = fmaxf(vmax, fabsf((float)u));
      }
    }
  } else if (live) {
    // singular line of the zero-flux Laplacian (Eq. 28 reading): project the
    // right-hand side to zero M_z-weighted mean, pin u_0 = 0, solve rows 1..nz-1,
    // then remove the weighted mean of the solution.
    double* cs = a.cs + off;
    double sm = 0.0, sf = 0.0;
    for (int k = 0; k < nz; ++k) {
      sm += s_m[k];
      sf += s_m[k] * (double)in[k * ks];
    }
    const double mu = sf / sm;
    double cprev = 0.0, dprev = 0.0;
    for (int k = 1; k < nz; ++k) {
      const double lo = (k > 1) ? -s_lo[k - 1] : 0.0;
      const double up = (k + 1 < nz) ? -s_lo[k] : 0.0;
      const double di = s * s_m[k] - lam * a.kdz[k];
      const double inv = 1.0 / (di - lo * cprev);
      cprev = up * inv;
      dprev = (s_m[k] * ((double)in[k * ks] - mu) - lo * dprev) * inv;
      cs[k * ks] = cprev;
      out[k * ks] = (T)dprev;
    }
    double u = dprev, su = s_m[nz - 1] * dprev;
    for (int k = nz - 2; k >= 1; --k) {
      u = (double)out[k * ks] - cs[k * ks] * u;
      out[k * ks] = (T)u;
      su += s_m[k] * u;
    }
    out[0] = (T)0.0;
    const double mean = su / sm;
    for (int k = 0; k < nz; ++k) {
      const double w = (double)out[k * ks] - mean;
      out[k * ks] = (T)w;
      vmax = fmaxf(vmax, fabsf((float)w));
    }
  }
  // one reduction point for the whole warp
  if (a.fmax) warp_max_out(vmax, a.fmax);
}

// the factors now in the cache belong to (sigma, lambda, field)
__global__ void k_thomas_key(double* key, double sigma, double lambda, int field, const int* __restrict__ skip) {
  if (skip && *skip) return;
  key[0] = sigma;
  key[1] = lambda;
  key[2] = (double)field;
}

__global__ void k_divide_f64(double* __restrict__ data, int nx, int ny, int nz, const double* __restrict__ lx,
                             const double* __restrict__ ly, const double* __restrict__ lz, double sigma,
                             double lambda, int singular_possible, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const long long P = (long long)nx * ny * nz;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.x * blockDim.x) {
    int i = (int)(p % nx);
    long long t = p / nx;
    int j = (int)(t % ny), k = (int)(t / ny);
    double ls = lx[i] + ly[j] + lz[k];
    double dv = sigma - lambda * ls;
    data[p] = (singular_possible && ls == 0.0) ? 0.0 : data[p] / dv;
  }
}

// cylindrical TPF (Eq. 46): data [k][j][i] with k the radial mode of theta
// mode j; u /= sigma - lam (Lx_i + Lr_{j,k})
__global__ void k_divide_modes_f64(double* __restrict__ data, int nx, int ny, int nz, const double* __restrict__ lx,
                                   const double* __restrict__ lr, double sigma, double lambda,
                                   const int* __restrict__ skip) {
  if (skip && *skip) return;
  const long long P = (long long)nx * ny * nz;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(p % nx);
    const long long t = p / nx;
    const int j = (int)(t % ny), k = (int)(t / ny);
    data[p] = data[p] / (sigma - lambda * (lx[i] + lr[(long long)j * nz + k]));
  }
}

struct StencilArgs {
  int nx, ny, nz;
  const double* wp[3];
  const double* wm[3];
  const double* w0[3];
  const double* m[3];
  const double* wyk;  // periodic y with the flux weight wyk[k] of plane k (cylindrical theta); null otherwise
};

__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh) {
#pragma unroll
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
    for (int q = 0; q < (int)(blockDim.x / 32); ++q) {
      sa += sh[2 * q];
      sb += sh[2 * q + 1];
    }
    a = sa;
    b = sb;
  }
}

__global__ void __launch_bounds__(kResThreads) k_residual_f64(StencilArgs g, const double* __restrict__ b,
                                                              const double* __restrict__ u, double* __restrict__ r,
                                                              double sigma, double lambda,
                                                              const DevStatus* __restrict__ st, int sub_mean,
                                                              double* __restrict__ partials,
                                                              const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double sh[2 * (kResThreads / 32)];
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long long sx = 1, sy = nx, sz = (long long)nx * ny;
  const long long P = sz * nz;
  const double mb = sub_mean ? st->mean_b : 0.0;
  double srr = 0.0, sbb = 0.0;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.x * blockDim.x) {
    int i = (int)(p % nx);
    long long t = p / nx;
    int j = (int)(t % ny), k = (int)(t / ny);
    double uc = u[p];
    double lx = g.w0[0][i] * uc, ly = 0.0, lz = g.w0[2][k] * uc;
    if (i + 1 < nx) lx += g.wp[0][i] * (u[p + sx] - uc);
    if (i > 0) lx += g.wm[0][i] * (u[p - sx] - uc);
    if (g.wyk) {
      const long long pn = j + 1 < ny ? p + sy : p - (ny - 1) * sy;
      const long long ps = j > 0 ? p - sy : p + (ny - 1) * sy;
      ly = g.wyk[k] * ((u[pn] - uc) + (u[ps] - uc));
    } else {
      ly = g.w0[1][j] * uc;
      if (j + 1 < ny) ly += g.wp[1][j] * (u[p + sy] - uc);
      if (j > 0) ly += g.wm[1][j] * (u[p - sy] - uc);
    }
    if (k + 1 < nz) lz += g.wp[2][k] * (u[p + sz] - uc);
    if (k > 0) lz += g.wm[2][k] * (u[p - sz] - uc);
    double bb = b[p] - mb;
    double rr = bb - (sigma * uc - lambda * ((lx + ly) + lz));
    if (r) r[p] = rr;
    srr += rr * rr;
    sbb += bb * bb;
  }
  block_sum2(srr, sbb, sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = srr;
    partials[2 * blockIdx.x + 1] = sbb;
  }
}

__global__ void k_finish_residual(const double* __restrict__ partials, int nblocks, DevStatus* st, double tol,
                                  int first, const int* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double sh[2 * 8];
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nblocks; q += blockDim.x) {
    a += partials[2 * q];
    b += partials[2 * q + 1];
  }
  block_sum2(a, b, sh);
  if (threadIdx.x == 0) {
    double rel = (b > 0.0) ? sqrt(a / b) : sqrt(a);
    if (first) {
      st->refine_steps = 0;
      st->bnorm2 = b;
    } else {
      st->refine_steps += 1;
    }
    st->rel_res = rel;
    if (first && !isfinite(b)) {
      st->error = 7;  // non-finite right-hand side
      st->done = 1;
    } else if (!isfinite(rel)) {
      st->error = 1;
      st->done = 1;
    } else {
      st->done = rel <= tol ? 1 : 0;
    }
  }
}

__global__ void __launch_bounds__(kResThreads) k_vmean_partial(StencilArgs g, const double* __restrict__ b,
                                                               double* __restrict__ partials) {
  __shared__ double sh[2 * (kResThreads / 32)];
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const long long P = (long long)nx * ny * nz;
  double sv = 0.0, sd = 0.0;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P;
       p += (long long)gridDim.x * blockDim.x) {
    int i = (int)(p % nx);
    long long t = p / nx;
    int j = (int)(t % ny), k = (int)(t / ny);
    double v = g.m[0][i] * g.m[1][j] * g.m[2][k];
    sv += v * b[p];
    sd += v;
  }
  block_sum2(sv, sd, sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = sv;
    partials[2 * blockIdx.x + 1] = sd;
  }
}

__global__ void k_vmean_finish(const double* __restrict__ partials, int nblocks, DevStatus* st) {
  __shared__ double sh[2 * 8];
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nblocks; q += blockDim.x) {
    a += partials[2 * q];
    b += partials[2 * q + 1];
  }
  block_sum2(a, b, sh);
  if (threadIdx.x == 0) st->mean_b = a / b;
}

__global__ void k_reset_status(DevStatus* st, double tol) {
  st->tol_used = tol;
  st->done = 0;
  st->refine_steps = 0;
  st->iters = 0;
  st->error = 0;
  st->rel_res = 0.0;
  st->bnorm2 = 0.0;
  st->mean_b = 0.0;
}

StencilArgs stencil_args(const Field& f) {
  StencilArgs g;
  g.nx = f.n[0];
  g.ny = f.n[1];
  g.nz = f.n[2];
  for (int d = 0; d < 3; ++d) {
    g.wp[d] = f.ax[d]->wp;
    g.wm[d] = f.ax[d]->wm;
    g.w0[d] = f.ax[d]->w0;
    g.m[d] = f.ax[d]->m;
  }
  g.wyk = nullptr;
  return g;
}

}  // namespace

fdi_status launch_lines_f64(fdi_plan* p, const double* in, double* out, const double* T, int nin, int nout,
                            long long lines, bool accumulate, const int* skip, cudaStream_t s) {
  FDI_KTIMER(p, "transform_x_f64", s);
  dim3 grid((unsigned)((lines + TB - 1) / TB), (unsigned)((nout + TB - 1) / TB));
  if (accumulate)
    k_lines_f64<true><<<grid, 256, 0, s>>>(in, out, T, nin, nout, lines, skip);
  else
    k_lines_f64<false><<<grid, 256, 0, s>>>(in, out, T, nin, nout, lines, skip);
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

fdi_status launch_slab_f64(fdi_plan* p, const double* in, double* out, const double* T, int nin, int nout,
                           long long ncols, int batch, const int* skip, cudaStream_t s) {
  FDI_KTIMER(p, batch > 1 ? "transform_y_f64" : "transform_z_f64", s);
  dim3 grid((unsigned)((ncols + TB - 1) / TB), (unsigned)((nout + TB - 1) / TB), (unsigned)batch);
  k_slab_f64<<<grid, 256, 0, s>>>(in, out, T, nin, nout, ncols, ncols, (long long)nin * ncols,
                                  (long long)nout * ncols, 0LL, skip);
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

fdi_status launch_modes_f64(fdi_plan* p, const double* in, double* out, const double* T_all, int n, int nx,
                            int ny, const int* skip, cudaStream_t s) {
  // field [n][ny][nx]; for every y index j (a theta mode) the n x n matrix
  // T_all + j n^2 contracts the outer index
  FDI_KTIMER(p, "transform_r_modes_f64", s);
  dim3 grid((unsigned)((nx + TB - 1) / TB), (unsigned)((n + TB - 1) / TB), (unsigned)ny);
  k_slab_f64<<<grid, 256, 0, s>>>(in, out, T_all, n, n, nx, (long long)nx * ny, nx, nx, (long long)n * n, skip);
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

fdi_status launch_thomas_f64(fdi_plan* p, const Field& f, double sigma, double lambda, int field, const double* in,
                             double* out, double* scratch, const int* skip, cudaStream_t s) {
  FDI_KTIMER(p, "thomas_z_f64", s);
  ThomasArgs a{};
  a.in = in;
  a.out = out;
  a.cs = scratch;
  a.nx = f.n[0];
  a.ny = f.n[1];
  a.nz = f.n[2];
  a.mixed_layout = 0;
  a.pitch = f.n[0];
  a.kstride = (long long)f.n[0] * f.n[1];
  a.lamx = f.ax[0]->lam;
  a.lamy = f.ax[1]->lam;
  a.mz = f.ax[2]->m;
  a.kdz = f.ax[2]->kd;
  a.koz = f.ax[2]->ko;
  a.wy = p->cyl_wy;
  a.sigma = sigma;
  a.lambda = lambda;
  a.field = field;
  a.singular_possible = (sigma == 0.0 && f.zero_flux_all) ? 1 : 0;
  const long long NL = (long long)a.nx * a.ny;
  const bool cache = p->tf && p->tf_q >= f.P;
  if (cache) {
    a.q = NL;
    a.cinv = p->tf;
    a.ccp = p->tf + p->tf_q;
    a.key = p->tf + 2 * p->tf_q;
  }
  k_thomas_f64<double><<<(unsigned)((NL + 127) / 128), 128, 0, s>>>(a, skip);
  FDI_LAUNCH_CHECK(p);
  if (cache) {
    k_thomas_key<<<1, 1, 0, s>>>(p->tf + 2 * p->tf_q, sigma, lambda, field, skip);
    FDI_LAUNCH_CHECK(p);
  }
  return FDI_OK;
}

fdi_status launch_thomas_cached_f32(fdi_plan* p, const Field& f, double sigma, double lambda, int field, float* data,
                                    int pitch, long long plane, float* fmax, const int* skip, cudaStream_t s) {
  FDI_KTIMER(p, "thomas_z_f64rec", s);
  ThomasArgs a{};
  a.in = data;
  a.out = data;
  a.cs = nullptr;
  a.nx = f.n[0];
  a.ny = f.n[1];
  a.nz = f.n[2];
  a.mixed_layout = 1;
  a.pitch = pitch;
  a.kstride = plane;
  a.lamx = f.ax[0]->lam;
  a.lamy = f.ax[1]->lam;
  a.mz = f.ax[2]->m;
  a.kdz = f.ax[2]->kd;
  a.koz = f.ax[2]->ko;
  a.wy = p->cyl_wy;
  a.sigma = sigma;
  a.lambda = lambda;
  a.field = field;
  a.singular_possible = 0;  // the singular problem keeps the FP32 sweep's null-line kernel
  a.fmax = fmax;
  const long long NL = (long long)a.nx * a.ny;
  a.q = NL;
  a.cinv = p->tf;
  a.ccp = p->tf + p->tf_q;
  a.key = p->tf + 2 * p->tf_q;
  k_thomas_f64<float><<<(unsigned)((NL + 127) / 128), 128, 0, s>>>(a, skip);
  FDI_LAUNCH_CHECK(p);
  k_thomas_key<<<1, 1, 0, s>>>(p->tf + 2 * p->tf_q, sigma, lambda, field, skip);
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

fdi_status launch_divide_f64(fdi_plan* p, const Field& f, double sigma, double lambda, double* data,
                             const int* skip, cudaStream_t s) {
  FDI_KTIMER(p, "divide_f64", s);
  int sp = (sigma == 0.0 && f.zero_flux_all) ? 1 : 0;
  k_divide_f64<<<152 * 8, 256, 0, s>>>(data, f.n[0], f.n[1], f.n[2], f.ax[0]->lam, f.ax[1]->lam, f.ax[2]->lam,
                                      sigma, lambda, sp, skip);
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

fdi_status launch_divide_modes_f64(fdi_plan* p, const Field& f, double sigma, double lambda, double* data,
                                  const int* skip, cudaStream_t s) {
  FDI_KTIMER(p, "divide_f64", s);
  k_divide_modes_f64<<<152 * 8, 256, 0, s>>>(data, f.n[0], f.n[1], f.n[2], f.ax[0]->lam, p->cyl_lr, sigma, lambda,
                                            skip);
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

fdi_status launch_residual_f64(fdi_plan* p, const Field& f, double sigma, double lambda, const double* b,
                               const double* u, double* r, bool subtract_mean, const int* skip,
                               cudaStream_t s) {
  FDI_KTIMER(p, "residual_f64", s);
  StencilArgs g = stencil_args(f);
  g.wyk = p->cyl_wres;
  k_residual_f64<<<kResBlocks, kResThreads, 0, s>>>(g, b, u, r, sigma, lambda, p->d_status, subtract_mean ? 1 : 0,
                                                    p->partials, skip);
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

fdi_status launch_finish_residual(fdi_plan* p, int nblocks, bool first, int /*count_step*/, const int* skip,
                                  cudaStream_t s) {
  FDI_KTIMER(p, "reduce", s);
  if (nblocks <= 0) nblocks = kResBlocks;
  k_finish_residual<<<1, 256, 0, s>>>(p->partials, nblocks, p->d_status, p->tol, first ? 1 : 0, skip);
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

fdi_status launch_mean_f64(fdi_plan* p, const Field& f, const double* b, cudaStream_t s) {
  FDI_KTIMER(p, "mean_f64", s);
  k_vmean_partial<<<kResBlocks, kResThreads, 0, s>>>(stencil_args(f), b, p->partials);
  FDI_LAUNCH_CHECK(p);
  k_vmean_finish<<<1, 256, 0, s>>>(p->partials, kResBlocks, p->d_status);
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

fdi_status launch_reset_status(fdi_plan* p, cudaStream_t s) {
  k_reset_status<<<1, 1, 0, s>>>(p->d_status, p->tol);
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

}  // namespace fdi
