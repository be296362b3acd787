// Mixed-precision Helmholtz / Laplace inverse: TPT with the x and y transforms
// on the tensor cores (split fp16, FP32 accumulation), the z Thomas sweep in
// FP32, and iterative refinement against a double-float residual.
//
// One direct solve (Sec. 3, TPT at the end of the section) is five passes over
// the field.  Each pass writes its output in the orientation the next pass
// reads with the contraction index contiguous:
//   r    [z][y][x]   residual (FP32), input of the forward x transform
//   F1   [z][i][y]   after E_x^{-1}   (i: x mode)
//   F2   [z][i][j]   after E_y^{-1}   (j: y mode); the Thomas sweep runs in place
//   F4   [z][y][i]   after E_y
//   H, L [z][y][x]   solution x = H + L in two FP32 planes: after the first
//                    solve H holds its output (exactly FP32); the first
//                    correction is stored as L (the pair is then exact, not
//                    renormalised); later corrections are added in
//                    double-float with renormalisation
// Rows are padded to a multiple of 4 floats (16-byte rows for vector loads).
//
// Refinement (the tensor-core solve is accurate to about 1e-6 relative):
//   r_0 = b;  H = S(r_0);  r_1 = b - A H;  L = S(r_1);
//   r_k = b - A (H + L) (double-float, flux form);  (H, L) += S(r_k)
//   until ||r_k|| / ||b|| <= tol.
// Every refinement-round kernel reads the device "done" flag and returns at
// once after convergence, so the solve is enqueued without host round trips.
#include <cmath>
#include <vector>

#include "df.cuh"
#include "fdi_internal.h"
#include "resid.cuh"
#include "resident.h"
#include "tc_transform.h"

namespace fdi {

struct MixedAxis {
  TcMatrix fwd, bwd;      // E^{-1} and E on the tensor cores
  float* m_f = nullptr;   // M, K of the Thomas direction in FP32
  float* kd_f = nullptr;
  float* ko_f = nullptr;
  float2* wp = nullptr;   // residual flux weights in double-float
  float2* wm = nullptr;
  float2* w0 = nullptr;
  float2* m_df = nullptr; // control-volume widths in double-float
  // resident solve (n <= 128): fwd and bwd in the shared-memory layout of its
  // MMAs (see tc_resident_image)
  uint8_t* rimg[2] = {nullptr, nullptr};
};

namespace {

constexpr int kBlocks = 152 * 8;
constexpr int kThreads = 256;
// per refinement round, the max |value| of each pass input: [0] r, [1] F1,
// [2] the z step's output, [3] F4, [4] F2 and [5] the divided spectrum (TPF)
constexpr int kScaleStride = 8;

int pitch4(int n) { return (n + 3) / 4 * 4; }

__device__ void finish_if_last(const FinishArgs& f, int t, int nt);

// The correction residual (MODE 1) takes the plain FP32 body when the first
// residual of this solve was small enough for the tolerance (a.fast_limit,
// set by the host; the first check records ||r_1|| / ||b|| in st->scal[1]);
// the choice is uniform over the grid.
template <int MODE, int SIG, bool LO, bool MEAN, bool OUT, bool CYL, bool VEC>
// occupancy: 3 CTAs per SM (80 registers) for the first residual; 4 (64) for
// the correction residual, whose usual body is the plain FP32 one (latency
// bound: more warps in flight), its exact body spilling a little
__global__ void __launch_bounds__(kResTX * kResTY, MODE == 1 ? 4 : 3) k_resid_df(ResidArgs a,
                                                                              const int* __restrict__ skip) {
  pdl_wait();
  if (skip && *skip) return;
  __shared__ double sh[4 * kResTY];
  const long long bid = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  if (MODE == 1 && !MEAN && a.fast_limit > 0.0 && a.st->scal[1] <= a.fast_limit)
    resid_body<MODE, SIG, LO, MEAN, OUT, CYL, VEC, true>(a, sh, blockIdx.x, blockIdx.y, blockIdx.z, bid);
  else
    resid_body<MODE, SIG, LO, MEAN, OUT, CYL, VEC, false>(a, sh, blockIdx.x, blockIdx.y, blockIdx.z, bid);
  finish_if_last(a.fin, threadIdx.y * kResTX + threadIdx.x, kResTX * kResTY);
}

using ResidKernel = void (*)(ResidArgs, const int*);

template <int SIG, bool CYL, bool VEC>
ResidKernel resid_kernel_s(int mode, bool lo, bool mean, bool out) {
  if (mode == 0)
    return mean ? k_resid_df<0, SIG, false, true, false, false, VEC> : k_resid_df<0, SIG, false, false, false, CYL, VEC>;
  if (mean)
    return lo ? k_resid_df<1, SIG, true, true, false, false, VEC> : k_resid_df<1, SIG, false, true, false, false, VEC>;
  if (out) return lo ? k_resid_df<1, SIG, true, false, true, CYL, VEC> : k_resid_df<1, SIG, false, false, true, CYL, VEC>;
  return lo ? k_resid_df<1, SIG, true, false, false, CYL, VEC> : k_resid_df<1, SIG, false, false, false, CYL, VEC>;
}

template <bool CYL, bool VEC>
ResidKernel resid_kernel_c(int sig_mode, int mode, bool lo, bool mean, bool out) {
  if (sig_mode == 0) return resid_kernel_s<0, CYL, VEC>(mode, lo, mean, out);
  if (sig_mode == 1) return resid_kernel_s<1, CYL, VEC>(mode, lo, mean, out);
  return resid_kernel_s<2, CYL, VEC>(mode, lo, mean, out);
}

// mode 0: r_1 = b - A H;  mode 1: r = r_1 - A L (lo: L has a low plane);
// cyl: periodic y with per-plane y weights (never singular, so no mean);
// vec: pairs moved by vector accesses (nx even, FP64 arrays 16-byte aligned)
ResidKernel resid_kernel(int sig_mode, int mode, bool lo, bool mean, bool out, bool cyl, bool vec) {
  if (cyl) return vec ? resid_kernel_c<true, true>(sig_mode, mode, lo, mean, out)
                      : resid_kernel_c<true, false>(sig_mode, mode, lo, mean, out);
  return vec ? resid_kernel_c<false, true>(sig_mode, mode, lo, mean, out)
             : resid_kernel_c<false, false>(sig_mode, mode, lo, mean, out);
}

// FP64 solution from the double-float accumulator (minus the volume-weighted
// mean for the zero-flux Laplace problem).
__global__ void k_finalize_out(const float* __restrict__ xh, const float* __restrict__ xl,
                               const float* __restrict__ xll, double* __restrict__ out, long long P,
                               const DevStatus* __restrict__ st, int max_refine, int singular) {
  pdl_wait();
  // refinement passes write the output themselves: only convergence in round 0
  // (no refinement step taken, L = 0) and the singular problem need this pass
  if (!singular && (st->refine_steps > 0 || max_refine == 0)) return;
  const bool has_l = st->refine_steps > 0, has_ll = st->refine_steps > 1;
  df::F2 mu = df::make(0.f, 0.f);
  if (singular) mu = df::from_f64(st->scal[0]);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
    df::F2 u = df::two_sum(xh[p], has_l ? xl[p] : 0.f);
    if (has_ll) u = df::fast_two_sum(u.hi, u.lo + xll[p]);
    if (singular) u = df::sub(u, mu);
    out[p] = df::to_f64_bits(u);
  }
}

// r_0 = b: FP64 -> FP32 copy into the padded residual layout, ||b||^2, max |b|
// and (singular problems) the volume-weighted sums; one warp per x-line
__global__ void __launch_bounds__(256) k_init_rhs(ResidArgs a) {
  pdl_wait();
  __shared__ double sh[4 * 8];
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int nwarps = gridDim.x * 8;
  float sbb = 0.f, rmax = 0.f;
  df::F2 svb = df::make(0.f, 0.f), sv = df::make(0.f, 0.f);
  for (int L = blockIdx.x * 8 + warp; L < ny * nz; L += nwarps) {
    const int j = L % ny, k = L / ny;
    const double* bl = a.b + (long long)L * nx;
    float* rl = a.r + ((long long)k * ny + j) * a.r_pitch;
    df::F2 Vjk = df::make(0.f, 0.f);
    if (a.want_mean) Vjk = df::mul(ld2(a.m[1] + j), ld2(a.m[2] + k));
    for (int i0 = 0; i0 < nx; i0 += 128) {
      double v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * 32 + lane;
        v[u] = i < nx ? bl[i] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * 32 + lane;
        if (i < nx) {
          const df::F2 bb = df::from_f64(v[u]);
          const float rf = bb.hi + bb.lo;
          rl[i] = rf;
          sbb = fmaf(rf, rf, sbb);
          rmax = fmaxf(rmax, fabsf(rf));
          if (a.want_mean) {
            const df::F2 V = df::mul(Vjk, ld2(a.m[0] + i));
            svb = df::add(svb, df::mul(V, bb));
            sv = df::add(sv, V);
          }
        }
      }
    }
  }
  double w[4] = {0.0, (double)sbb, df::to_f64(svb), df::to_f64(sv)};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int q = 0; q < 4; ++q) w[q] += __shfl_down_sync(0xffffffffu, w[q], o);
    rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  }
  if (lane == 0) {
    for (int q = 0; q < 4; ++q) sh[4 * warp + q] = w[q];
    if (rmax > 0.f) atomicMax(reinterpret_cast<unsigned int*>(a.rmax), __float_as_uint(rmax));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[4] = {0, 0, 0, 0};
    for (int q = 0; q < 8; ++q)
      for (int c = 0; c < 4; ++c) t[c] += sh[4 * q + c];
    for (int c = 0; c < 4; ++c) a.partials[4 * blockIdx.x + c] = t[c];
  }
  finish_if_last(a.fin, threadIdx.x, blockDim.x);
}

// r_0 = b for unpadded fields without the mean (nx a multiple of 4): flat
// stream, 8 values per thread and iteration (four 16-byte loads in flight),
// ||b||^2 and max |b|
__global__ void __launch_bounds__(256) k_init_rhs_flat(ResidArgs a, long long P) {
  pdl_wait();
  __shared__ double sh[8];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  float sbb = 0.f, rmax = 0.f;
  const long long stride = (long long)gridDim.x * blockDim.x * 8;
  for (long long p0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 8; p0 < P; p0 += stride) {
    double v[8];
    if (p0 + 8 <= P) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double2 t = *reinterpret_cast<const double2*>(a.b + p0 + 2 * u);
        v[2 * u] = t.x;
        v[2 * u + 1] = t.y;
      }
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = p0 + u < P ? a.b[p0 + u] : 0.0;
    }
    float f[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const df::F2 bb = df::from_f64(v[u]);
      f[u] = bb.hi + bb.lo;
      sbb = fmaf(f[u], f[u], sbb);
      rmax = fmaxf(rmax, fabsf(f[u]));
    }
    if (p0 + 8 <= P) {
      *reinterpret_cast<float4*>(a.r + p0) = make_float4(f[0], f[1], f[2], f[3]);
      *reinterpret_cast<float4*>(a.r + p0 + 4) = make_float4(f[4], f[5], f[6], f[7]);
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (p0 + u < P) a.r[p0 + u] = f[u];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sbb += __shfl_down_sync(0xffffffffu, sbb, o);
    rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  }
  if (lane == 0) {
    sh[warp] = (double)sbb;
    if (rmax > 0.f) atomicMax(reinterpret_cast<unsigned int*>(a.rmax), __float_as_uint(rmax));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += sh[q];
    a.partials[4 * blockIdx.x + 0] = 0.0;
    a.partials[4 * blockIdx.x + 1] = t;
    a.partials[4 * blockIdx.x + 2] = 0.0;
    a.partials[4 * blockIdx.x + 3] = 0.0;
  }
  finish_if_last(a.fin, threadIdx.x, blockDim.x);
}

// lambda-scaled double-float flux weights of the three directions
__global__ void k_scale_weights(const float2* __restrict__ wp0, const float2* __restrict__ wm0,
                                const float2* __restrict__ w00, int n0, const float2* __restrict__ wp1,
                                const float2* __restrict__ wm1, const float2* __restrict__ w01, int n1,
                                const float2* __restrict__ wp2, const float2* __restrict__ wm2,
                                const float2* __restrict__ w02, int n2, const float2* __restrict__ wc, int nc,
                                float2 lam, float2* __restrict__ out) {
  // out layout: [3 directions][3 kinds (p, m, 0)][kMaxN], then (cylindrical
  // plans, block 9) the theta flux weight per radial cell
  if (blockIdx.x == 9) {
    for (int t = threadIdx.x; t < nc; t += blockDim.x) {
      const df::F2 v = df::mul(df::make(lam.x, lam.y), ld2(wc + t));
      out[9 * kMaxN + t] = make_float2(v.hi, v.lo);
    }
    return;
  }
  const int d = blockIdx.x / 3, kind = blockIdx.x % 3;
  const int n = d == 0 ? n0 : (d == 1 ? n1 : n2);
  const float2* src = d == 0 ? (kind == 0 ? wp0 : kind == 1 ? wm0 : w00)
                             : d == 1 ? (kind == 0 ? wp1 : kind == 1 ? wm1 : w01)
                                      : (kind == 0 ? wp2 : kind == 1 ? wm2 : w02);
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const df::F2 v = df::mul(df::make(lam.x, lam.y), ld2(src + t));
    out[(d * 3 + kind) * kMaxN + t] = make_float2(v.hi, v.lo);
  }
}

// The last block of a reduction grid to finish (atomic ticket after its
// partials are visible) runs finish_block and re-arms the ticket counter, so
// the reduction needs no second launch.  Every block has passed its own skip
// test before the last one can change the done flag.
__device__ void finish_if_last(const FinishArgs& f, int t, int nt) {
  __shared__ int amlast;
  const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
  if (t == 0) {
    __threadfence();
    amlast = atomicAdd(f.counter, 1u) == nb - 1 ? 1 : 0;
  }
  __syncthreads();
  if (!amlast) return;
  __threadfence();
  finish_block(f.partials, (int)nb, f.st, f.tol, f.kind, f.want_mean, t, nt);
  if (t == 0) {
    *f.counter = 0u;
    if (f.next_round) cudaGraphSetConditional(f.next_round, f.st->done ? 0u : 1u);
  }
}

struct Thomas32Args {
  float* f;           // in/out, element (z, i, j) at z*plane + i*pitch + j
  float* cs;          // scratch c'_k, same layout
  int nx, ny, nz, pitch;
  long long plane;
  const double* lamx;
  const double* lamy;
  const float* mz;
  const float* kdz;
  const float* koz;
  const float* wy;    // cylindrical plans: per z weight of the y (theta) eigenvalue, A_i g_i
  double sigma, lambda;
  int singular_possible;
  float* fmax;
};

// diagonal of step k of the line sweep: s M_k - lambda Kd_k, and on
// cylindrical plans also ly * swy_k with ly = -Lambda_y of the line and
// swy_k = lambda wy_k (s then holds sigma - lambda Lambda_x only)
template <bool CYL>
__device__ __forceinline__ float thomas_diag(float s, float ly, float4 co, const float* swy, int k) {
  return CYL ? fmaf(s, co.x, fmaf(ly, swy[k], -co.y)) : fmaf(s, co.x, -co.y);
}

constexpr int kTB = 16;   // Thomas block of planes: c' checkpoint interval and copy group
constexpr int kNBR = 3;   // blocks of kTB planes in flight per line

// single-instruction reciprocal (PTX rcp.approx, at most 1 ulp): the sweep
// only needs FP32 accuracy, the refinement restores the rest
__device__ __forceinline__ float rcp_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// one elimination step of the z sweep: c'_k and d'_k from c'_{k-1}, d'_{k-1}
__device__ __forceinline__ void thomas_step(float s, float m, float lkd, float lo, float up, float f, float& cp,
                                            float& dp) {
  const float di = fmaf(s, m, -lkd);
  const float inv = rcp_fast(fmaf(-lo, cp, di));
  cp = up * inv;
  dp = fmaf(m, f, -lo * dp) * inv;
}

// per-thread asynchronous 4-byte copies global -> shared (each thread reads
// back only its own slots, so completion is tracked per thread by groups)
__device__ __forceinline__ void cp_async4(unsigned dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// TL: lines per CTA (one thread per line; a tuning knob).  FULL: nz is a
// multiple of kTB (no partial block of planes)
template <int TL, bool FULL, bool CYL>
__global__ void __launch_bounds__(TL) k_thomas_f32(Thomas32Args a, const int* __restrict__ skip) {
  constexpr int kTL = TL;
  pdl_wait();
  if (skip && *skip) return;
  // coefficients of the z operator in shared memory: {M_k, lambda Kd_k,
  // lower, upper} with the off-diagonals negated (lambda-scaled), and the
  // per-thread ring of planes in flight and c' checkpoints
  __shared__ float4 s_co[kMaxN];
  __shared__ float s_m[kMaxN], s_lkd[kMaxN], s_lko[kMaxN + 1];
  __shared__ float ring[kNBR * kTB][kTL];
  __shared__ float ckp[kMaxN / kTB][kTL];
  __shared__ float s_wy[CYL ? kMaxN : 1];
  const int nz = a.nz;
  const float lam = (float)a.lambda;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    const float lko_k = (k + 1 < nz) ? lam * a.koz[k] : 0.f;
    const float lko_m = (k > 0) ? lam * a.koz[k - 1] : 0.f;
    s_co[k] = make_float4(a.mz[k], lam * a.kdz[k], -lko_m, -lko_k);
    s_m[k] = a.mz[k];
    s_lkd[k] = lam * a.kdz[k];
    s_lko[k] = lko_k;
    if (CYL) s_wy[k] = lam * a.wy[k];
  }
  __syncthreads();
  const int tid = threadIdx.x;
  const long long t = (long long)blockIdx.x * blockDim.x + tid;
  float vmax = 0.f;
  if (t < (long long)a.nx * a.ny) {
    const int i = (int)(t / a.ny), j = (int)(t % a.ny);
    const int pl = (int)a.plane;  // plane stride in elements (< 2^31 / kMaxN)
    const double lab = a.lamx[i] + a.lamy[j];
    const float s = (float)(a.sigma - a.lambda * (CYL ? a.lamx[i] : lab));
    const float ly = CYL ? (float)(-a.lamy[j]) : 0.f;
    float* f = a.f + (long long)i * a.pitch + j;
    if (!(a.singular_possible && lab == 0.0)) {
      const int nb = (nz + kTB - 1) / kTB;
      const unsigned ring0 = (unsigned)__cvta_generic_to_shared(&ring[0][tid]);
      // request block b of planes into its ring slot (one copy group per block)
      auto fetch = [&](int b) {
        if (b >= 0 && b < nb) {
          const unsigned dst = ring0 + (unsigned)((b % kNBR) * kTB * kTL * 4);
          const float* src = f + (long long)b * kTB * pl;
          const int cnt = FULL ? kTB : min(kTB, nz - b * kTB);
#pragma unroll
          for (int e = 0; e < kTB; ++e)
            if (FULL || e < cnt) cp_async4(dst + e * kTL * 4, src + e * pl);
        }
        cp_async_commit();
      };
      // forward elimination: d'_k stored in place, c'_{k-1} kept at each block start
      for (int q = 0; q < kNBR - 1; ++q) fetch(q);
      float cp = 0.f, dp = 0.f;
      for (int b = 0; b < nb; ++b) {
        fetch(b + kNBR - 1);
        cp_async_wait<kNBR - 1>();
        ckp[b][tid] = cp;
        const float* rs = &ring[(b % kNBR) * kTB][tid];
        float* fo = f + (long long)b * kTB * pl;
        const int k0 = b * kTB;
#pragma unroll
        for (int e = 0; e < kTB; ++e) {
          if (FULL || k0 + e < nz) {
            const float4 co = s_co[k0 + e];
            const float inv = rcp_fast(fmaf(-co.z, cp, thomas_diag<CYL>(s, ly, co, s_wy, k0 + e)));
            cp = co.w * inv;
            dp = fmaf(co.x, rs[e * kTL], -co.z * dp) * inv;
            fo[e * pl] = dp;
          }
        }
      }
      cp_async_wait<0>();
      // back substitution from the top, streaming d' block by block in
      // reverse; c'_k is recomputed from the checkpoint with the same
      // operations (bit-identical).  The top plane has c' = 0 (no upper
      // neighbour), so u_{nz-1} = d'_{nz-1} falls out of the same update.
      for (int q = 0; q < kNBR - 1; ++q) fetch(nb - 1 - q);
      float u = 0.f;
      for (int b = nb - 1; b >= 0; --b) {
        fetch(b - (kNBR - 1));
        const int k0 = b * kTB;
        float cpb[kTB];
        float c = ckp[b][tid];
#pragma unroll
        for (int e = 0; e < kTB; ++e) {
          if (FULL || k0 + e < nz) {
            const float4 co = s_co[k0 + e];
            c = co.w * rcp_fast(fmaf(-co.z, c, thomas_diag<CYL>(s, ly, co, s_wy, k0 + e)));
          }
          cpb[e] = c;
        }
        cp_async_wait<kNBR - 1>();
        const float* rs = &ring[(b % kNBR) * kTB][tid];
        float* fo = f + (long long)k0 * pl;
#pragma unroll
        for (int e = kTB - 1; e >= 0; --e) {
          if (FULL || k0 + e < nz) {
            u = fmaf(-cpb[e], u, rs[e * kTL]);
            fo[e * pl] = u;
            vmax = fmaxf(vmax, fabsf(u));
          }
        }
      }
      cp_async_wait<0>();
    } else {
      // singular line of the zero-flux Laplacian: project, pin u_0 = 0, solve, re-centre
      float* cs = a.cs + (long long)i * a.pitch + j;
      float sm = 0.f, sf = 0.f;
      for (int k = 0; k < nz; ++k) {
        sm += s_m[k];
        sf = fmaf(s_m[k], f[k * pl], sf);
      }
      const float mu = sf / sm;
      float cp = 0.f, dp = 0.f;
      for (int k = 1; k < nz; ++k) {
        const float lo = k > 1 ? -s_lko[k - 1] : 0.f;
        thomas_step(s, s_m[k], s_lkd[k], lo, -s_lko[k], f[k * pl] - mu, cp, dp);
        cs[k * pl] = cp;
        f[k * pl] = dp;
      }
      float u = dp, su = s_m[nz - 1] * dp;
      for (int k = nz - 2; k >= 1; --k) {
        u = fmaf(-cs[k * pl], u, f[k * pl]);
        f[k * pl] = u;
        su = fmaf(s_m[k], u, su);
      }
      f[0] = 0.f;
      const float mean = su / sm;
      for (int k = 0; k < nz; ++k) {
        const float w = f[k * pl] - mean;
        f[k * pl] = w;
        vmax = fmaxf(vmax, fabsf(w));
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  if ((threadIdx.x & 31) == 0 && vmax > 0.f) atomicMax(reinterpret_cast<unsigned int*>(a.fmax), __float_as_uint(vmax));
}

__device__ __forceinline__ void cp_async8(unsigned dst, const float2* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}

// FP32 Thomas sweep, two adjacent lines (i, j) and (i, j + 1) per thread (j
// even): the copies, shared-memory reads, stores and coefficient reads are
// shared by the two recurrences, which also give the thread two independent
// dependency chains.  A pair holding the singular line of the zero-flux
// Laplacian is left to k_thomas_f32 (launched over that pair only).  When ny
// is odd the last pair's second line is a padding column of the row: it is
// swept with a valid eigenvalue and excluded from the scale.
// The forward elimination stores nothing but c' and d' at the block
// boundaries (shared memory); the back substitution reads f again and
// recomputes c' and d' of each block of kTB planes from its boundary values,
// with the forward pass's arithmetic (so the same values), before it runs the
// block downwards.  Per point that is f read twice and u written once (12
// bytes) instead of f read, d' written and read back, u written (16 bytes);
// the top kNBR blocks are still in the copy ring when the back substitution
// starts and are not read again.
template <int TL, bool FULL, bool CYL>
__global__ void __launch_bounds__(TL) k_thomas2_f32(Thomas32Args a, const int* __restrict__ skip) {
  pdl_wait();
  if (skip && *skip) return;
  __shared__ float4 s_co[kMaxN];
  __shared__ float2 ring[kNBR * kTB][TL];
  __shared__ float2 ckp[kMaxN / kTB][TL];
  __shared__ float2 dkp[kMaxN / kTB][TL];
  __shared__ float s_wy[CYL ? kMaxN : 1];
  const int nz = a.nz;
  const float lam = (float)a.lambda;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    const float lko_k = (k + 1 < nz) ? lam * a.koz[k] : 0.f;
    const float lko_m = (k > 0) ? lam * a.koz[k - 1] : 0.f;
    s_co[k] = make_float4(a.mz[k], lam * a.kdz[k], -lko_m, -lko_k);
    if (CYL) s_wy[k] = lam * a.wy[k];
  }
  __syncthreads();
  const int tid = threadIdx.x;
  const int npair = (a.ny + 1) / 2;
  const long long t = (long long)blockIdx.x * blockDim.x + tid;
  float vmax = 0.f;
  if (t < (long long)a.nx * npair) {
    const int i = (int)(t / npair), j0 = 2 * (int)(t % npair);
    const bool second = j0 + 1 < a.ny;
    const int pl2 = (int)(a.plane / 2);  // plane stride in float2 (plane and pitch are even)
    const double lab0 = a.lamx[i] + a.lamy[j0];
    const double lab1 = a.lamx[i] + a.lamy[second ? j0 + 1 : j0];
    if (!(a.singular_possible && (lab0 == 0.0 || lab1 == 0.0))) {
      const float s0 = (float)(a.sigma - a.lambda * (CYL ? a.lamx[i] : lab0));
      const float s1 = (float)(a.sigma - a.lambda * (CYL ? a.lamx[i] : lab1));
      const float ly0 = CYL ? (float)(-a.lamy[j0]) : 0.f;
      const float ly1 = CYL ? (float)(-a.lamy[second ? j0 + 1 : j0]) : 0.f;
      float2* f = reinterpret_cast<float2*>(a.f + (long long)i * a.pitch + j0);
      const int nb = (nz + kTB - 1) / kTB;
      const unsigned ring0 = (unsigned)__cvta_generic_to_shared(&ring[0][tid]);
      auto fetch = [&](int b) {
        if (b >= 0 && b < nb) {
          const unsigned dst = ring0 + (unsigned)((b % kNBR) * kTB * TL * 8);
          const float2* src = f + (long long)b * kTB * pl2;
          const int cnt = FULL ? kTB : min(kTB, nz - b * kTB);
#pragma unroll
          for (int e = 0; e < kTB; ++e)
            if (FULL || e < cnt) cp_async8(dst + e * TL * 8, src + e * pl2);
        }
        cp_async_commit();
      };
      for (int q = 0; q < kNBR - 1; ++q) fetch(q);
      float cp0 = 0.f, dp0 = 0.f, cp1 = 0.f, dp1 = 0.f;
      for (int b = 0; b < nb; ++b) {
        fetch(b + kNBR - 1);
        cp_async_wait<kNBR - 1>();
        ckp[b][tid] = make_float2(cp0, cp1);
        dkp[b][tid] = make_float2(dp0, dp1);
        const float2* rs = &ring[(b % kNBR) * kTB][tid];
        const int k0 = b * kTB;
#pragma unroll
        for (int e = 0; e < kTB; ++e) {
          if (FULL || k0 + e < nz) {
            const float4 co = s_co[k0 + e];
            const float2 fv = rs[e * TL];
            const float inv0 = rcp_fast(fmaf(-co.z, cp0, thomas_diag<CYL>(s0, ly0, co, s_wy, k0 + e)));
            const float inv1 = rcp_fast(fmaf(-co.z, cp1, thomas_diag<CYL>(s1, ly1, co, s_wy, k0 + e)));
            cp0 = co.w * inv0;
            cp1 = co.w * inv1;
            dp0 = fmaf(co.x, fv.x, -co.z * dp0) * inv0;
            dp1 = fmaf(co.x, fv.y, -co.z * dp1) * inv1;
          }
        }
      }
      cp_async_wait<0>();
      // blocks nb - kNBR .. nb - 1 are in the ring (f is not written above)
      auto refetch = [&](int b) {
        if (b < nb - kNBR) fetch(b);
        else cp_async_commit();
      };
      for (int q = 0; q < kNBR - 1; ++q) refetch(nb - 1 - q);
      float u0 = 0.f, u1 = 0.f;
      for (int b = nb - 1; b >= 0; --b) {
        refetch(b - (kNBR - 1));
        const int k0 = b * kTB;
        float cpb0[kTB], cpb1[kTB], dpb0[kTB], dpb1[kTB];
        const float2 cc = ckp[b][tid], dd = dkp[b][tid];
        float c0 = cc.x, c1 = cc.y, d0 = dd.x, d1 = dd.y;
        cp_async_wait<kNBR - 1>();
        const float2* rs = &ring[(b % kNBR) * kTB][tid];
#pragma unroll
        for (int e = 0; e < kTB; ++e) {
          if (FULL || k0 + e < nz) {
            const float4 co = s_co[k0 + e];
            const float2 fv = rs[e * TL];
            const float inv0 = rcp_fast(fmaf(-co.z, c0, thomas_diag<CYL>(s0, ly0, co, s_wy, k0 + e)));
            const float inv1 = rcp_fast(fmaf(-co.z, c1, thomas_diag<CYL>(s1, ly1, co, s_wy, k0 + e)));
            c0 = co.w * inv0;
            c1 = co.w * inv1;
            d0 = fmaf(co.x, fv.x, -co.z * d0) * inv0;
            d1 = fmaf(co.x, fv.y, -co.z * d1) * inv1;
          }
          cpb0[e] = c0;
          cpb1[e] = c1;
          dpb0[e] = d0;
          dpb1[e] = d1;
        }
        float2* fo = f + (long long)k0 * pl2;
#pragma unroll
        for (int e = kTB - 1; e >= 0; --e) {
          if (FULL || k0 + e < nz) {
            u0 = fmaf(-cpb0[e], u0, dpb0[e]);
            u1 = fmaf(-cpb1[e], u1, dpb1[e]);
            fo[e * pl2] = make_float2(u0, u1);
            vmax = fmaxf(vmax, fabsf(u0));
            if (second) vmax = fmaxf(vmax, fabsf(u1));
          }
        }
      }
      cp_async_wait<0>();
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  if ((threadIdx.x & 31) == 0 && vmax > 0.f) atomicMax(reinterpret_cast<unsigned int*>(a.fmax), __float_as_uint(vmax));
}

// The same two-lines-per-thread sweep keeping d' of the top kTopBlocks blocks
// of planes in shared memory: the forward sweep stores them there instead of
// in the field, and the back substitution, which starts at the top, reads them
// back without a round trip to HBM (8 bytes per point less for those planes;
// every plane for nz <= 128).  Arithmetic and results are those of
// k_thomas2_f32.  64 KB of dynamic shared memory per CTA.
constexpr int kTopBlocks = 8;
constexpr int kTopBytes = kTopBlocks * kTB * 64 * (int)sizeof(float2);

template <bool FULL, bool CYL>
__global__ void __launch_bounds__(64) k_thomas2c_f32(Thomas32Args a, const int* __restrict__ skip) {
  constexpr int TL = 64;
  pdl_wait();
  if (skip && *skip) return;
  __shared__ float4 s_co[kMaxN];
  __shared__ float2 ring[kNBR * kTB][TL];
  __shared__ float2 ckp[kMaxN / kTB][TL];
  __shared__ float s_wy[CYL ? kMaxN : 1];
  extern __shared__ float2 s_top[];  // [kTopBlocks * kTB][TL]
  const int nz = a.nz;
  const float lam = (float)a.lambda;
  for (int k = threadIdx.x; k < nz; k += blockDim.x) {
    const float lko_k = (k + 1 < nz) ? lam * a.koz[k] : 0.f;
    const float lko_m = (k > 0) ? lam * a.koz[k - 1] : 0.f;
    s_co[k] = make_float4(a.mz[k], lam * a.kdz[k], -lko_m, -lko_k);
    if (CYL) s_wy[k] = lam * a.wy[k];
  }
  __syncthreads();
  const int tid = threadIdx.x;
  const int npair = (a.ny + 1) / 2;
  const long long t = (long long)blockIdx.x * blockDim.x + tid;
  float vmax = 0.f;
  if (t < (long long)a.nx * npair) {
    const int i = (int)(t / npair), j0 = 2 * (int)(t % npair);
    const bool second = j0 + 1 < a.ny;
    const int pl2 = (int)(a.plane / 2);
    const double lab0 = a.lamx[i] + a.lamy[j0];
    const double lab1 = a.lamx[i] + a.lamy[second ? j0 + 1 : j0];
    if (!(a.singular_possible && (lab0 == 0.0 || lab1 == 0.0))) {
      const float s0 = (float)(a.sigma - a.lambda * (CYL ? a.lamx[i] : lab0));
      const float s1 = (float)(a.sigma - a.lambda * (CYL ? a.lamx[i] : lab1));
      const float ly0 = CYL ? (float)(-a.lamy[j0]) : 0.f;
      const float ly1 = CYL ? (float)(-a.lamy[second ? j0 + 1 : j0]) : 0.f;
      float2* f = reinterpret_cast<float2*>(a.f + (long long)i * a.pitch + j0);
      const int nb = (nz + kTB - 1) / kTB;
      const int gb = nb > kTopBlocks ? nb - kTopBlocks : 0;  // blocks below gb go through the field
      const unsigned ring0 = (unsigned)__cvta_generic_to_shared(&ring[0][tid]);
      auto fetch = [&](int b) {
        if (b >= 0 && b < nb) {
          const unsigned dst = ring0 + (unsigned)((b % kNBR) * kTB * TL * 8);
          const float2* src = f + (long long)b * kTB * pl2;
          const int cnt = FULL ? kTB : min(kTB, nz - b * kTB);
#pragma unroll
          for (int e = 0; e < kTB; ++e)
            if (FULL || e < cnt) cp_async8(dst + e * TL * 8, src + e * pl2);
        }
        cp_async_commit();
      };
      for (int q = 0; q < kNBR - 1; ++q) fetch(q);
      float cp0 = 0.f, dp0 = 0.f, cp1 = 0.f, dp1 = 0.f;
      for (int b = 0; b < nb; ++b) {
        fetch(b + kNBR - 1);
        cp_async_wait<kNBR - 1>();
        ckp[b][tid] = make_float2(cp0, cp1);
        const float2* rs = &ring[(b % kNBR) * kTB][tid];
        float2* fo = f + (long long)b * kTB * pl2;
        float2* to = &s_top[(b - gb) * kTB * TL + tid];
        const int k0 = b * kTB;
#pragma unroll
        for (int e = 0; e < kTB; ++e) {
          if (FULL || k0 + e < nz) {
            const float4 co = s_co[k0 + e];
            const float2 fv = rs[e * TL];
            const float inv0 = rcp_fast(fmaf(-co.z, cp0, thomas_diag<CYL>(s0, ly0, co, s_wy, k0 + e)));
            const float inv1 = rcp_fast(fmaf(-co.z, cp1, thomas_diag<CYL>(s1, ly1, co, s_wy, k0 + e)));
            cp0 = co.w * inv0;
            cp1 = co.w * inv1;
            dp0 = fmaf(co.x, fv.x, -co.z * dp0) * inv0;
            dp1 = fmaf(co.x, fv.y, -co.z * dp1) * inv1;
            if (b >= gb)
              to[e * TL] = make_float2(dp0, dp1);
            else
              fo[e * pl2] = make_float2(dp0, dp1);
          }
        }
      }
      cp_async_wait<0>();
      // back substitution: the on-chip blocks first, then the field's, whose
      // copies are requested kNBR - 1 blocks ahead
      for (int q = 0; q < kNBR - 1; ++q) fetch(gb - 1 - q);
      float u0 = 0.f, u1 = 0.f;
      for (int b = nb - 1; b >= 0; --b) {
        if (b < gb) fetch(b - (kNBR - 1));
        const int k0 = b * kTB;
        float cpb0[kTB], cpb1[kTB];
        const float2 cc = ckp[b][tid];
        float c0 = cc.x, c1 = cc.y;
#pragma unroll
        for (int e = 0; e < kTB; ++e) {
          if (FULL || k0 + e < nz) {
            const float4 co = s_co[k0 + e];
            c0 = co.w * rcp_fast(fmaf(-co.z, c0, thomas_diag<CYL>(s0, ly0, co, s_wy, k0 + e)));
            c1 = co.w * rcp_fast(fmaf(-co.z, c1, thomas_diag<CYL>(s1, ly1, co, s_wy, k0 + e)));
          }
          cpb0[e] = c0;
          cpb1[e] = c1;
        }
        const float2* rs;
        int rstride;
        if (b < gb) {
          cp_async_wait<kNBR - 1>();
          rs = &ring[(b % kNBR) * kTB][tid];
        } else {
          rs = &s_top[(b - gb) * kTB * TL + tid];
        }
        rstride = TL;
        float2* fo = f + (long long)k0 * pl2;
#pragma unroll
        for (int e = kTB - 1; e >= 0; --e) {
          if (FULL || k0 + e < nz) {
            const float2 dv = rs[e * rstride];
            u0 = fmaf(-cpb0[e], u0, dv.x);
            u1 = fmaf(-cpb1[e], u1, dv.y);
            fo[e * pl2] = make_float2(u0, u1);
            vmax = fmaxf(vmax, fabsf(u0));
            if (second) vmax = fmaxf(vmax, fabsf(u1));
          }
        }
      }
      cp_async_wait<0>();
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  if ((threadIdx.x & 31) == 0 && vmax > 0.f) atomicMax(reinterpret_cast<unsigned int*>(a.fmax), __float_as_uint(vmax));
}

// TPF spectral divide (Eq. 26-28 with sigma): f[k][i][j] /= sigma - lambda
// (Lambda_x,i + Lambda_y,j + Lambda_z,k) on the padded [nz][nx][py] layout
// (padding columns untouched), and max |result|.  The shifted eigenvalues are
// FP32 (every term has the same sign, so the sum loses nothing to
// cancellation); the null mode of the singular zero-flux Laplacian is set to 0.
// One warp per (k, i) row, four columns per lane and step.
__global__ void __launch_bounds__(256) k_divide_tpf(float* __restrict__ f, int nx, int ny, int py, int nz,
                                                    const double* __restrict__ lx, const double* __restrict__ ly,
                                                    const double* __restrict__ lz, double sigma, double lambda,
                                                    int singular, float* __restrict__ fmax,
                                                    const int* __restrict__ skip) {
  pdl_wait();
  if (skip && *skip) return;
  __shared__ float s_lx[kMaxN], s_ly[kMaxN], s_lz[kMaxN];
  for (int t = threadIdx.x; t < kMaxN; t += blockDim.x) {
    s_lx[t] = t < nx ? (float)(-lambda * lx[t]) : 0.f;
    s_ly[t] = t < ny ? (float)(-lambda * ly[t]) : 0.f;
    s_lz[t] = t < nz ? (float)(-lambda * lz[t]) : 0.f;
  }
  __syncthreads();
  const float sg = (float)sigma;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  float vmax = 0.f;
  for (long long row = (long long)blockIdx.x * 8 + warp; row < (long long)nz * nx; row += (long long)gridDim.x * 8) {
    const int i = (int)(row % nx), k = (int)(row / nx);
    const float base = sg + s_lx[i] + s_lz[k];
    float4* fr = reinterpret_cast<float4*>(f + row * py);
    for (int q = lane; q < py / 4; q += 32) {
      float4 v = fr[q];
      float* e = reinterpret_cast<float*>(&v);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = 4 * q + c;
        if (j < ny) {
          const float den = base + s_ly[j];
          e[c] = (singular && den == 0.f) ? 0.f : e[c] / den;
          vmax = fmaxf(vmax, fabsf(e[c]));
        }
      }
      fr[q] = v;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  if (lane == 0 && vmax > 0.f) atomicMax(reinterpret_cast<unsigned int*>(fmax), __float_as_uint(vmax));
}

__global__ void k_absmax(const float* __restrict__ in, long long rows, int n, int pitch, float* __restrict__ mx) {
  float v = 0.f;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < rows * n;
       q += (long long)gridDim.x * blockDim.x)
    v = fmaxf(v, fabsf(in[(q / n) * pitch + q % n]));
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0 && v > 0.f) atomicMax(reinterpret_cast<unsigned int*>(mx), __float_as_uint(v));
}

#define FDI_TRY(expr)            \
  do {                           \
    fdi_status _s = (expr);      \
    if (_s != FDI_OK) return _s; \
  } while (0)

float2 split_host(double v) {
  float h = (float)v;
  float l = (float)(v - (double)h);
  return make_float2(h, l);
}

fdi_status upload_df(float2** dst, const std::vector<double>& v) {
  std::vector<float2> h(v.size());
  for (size_t i = 0; i < v.size(); ++i) h[i] = split_host(v[i]);
  FDI_CUDA_TRY(cudaMalloc(dst, std::max<size_t>(1, h.size()) * sizeof(float2)));
  FDI_CUDA_TRY(cudaMemcpy(*dst, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice));
  return FDI_OK;
}

fdi_status upload_f(float** dst, const std::vector<double>& v) {
  std::vector<float> h(v.size());
  for (size_t i = 0; i < v.size(); ++i) h[i] = (float)v[i];
  FDI_CUDA_TRY(cudaMalloc(dst, std::max<size_t>(1, h.size()) * sizeof(float)));
  FDI_CUDA_TRY(cudaMemcpy(*dst, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
  return FDI_OK;
}

fdi_status setup_axis(fdi_plan* p, Axis* ax, cudaStream_t s) {
  MixedAxis* mx = new MixedAxis();
  ax->mixed = mx;
  const int n = ax->n;
  FDI_TRY(tc_prepare_matrix(p, ax->Einv, n, &mx->fwd, s));
  FDI_TRY(tc_prepare_matrix(p, ax->E, n, &mx->bwd, s));
  if (n <= kResMaxPlane) {
    FDI_TRY(tc_resident_image(p, mx->fwd, &mx->rimg[0], s));
    FDI_TRY(tc_resident_image(p, mx->bwd, &mx->rimg[1], s));
  }
  FDI_TRY(upload_f(&mx->m_f, ax->h_m));
  FDI_TRY(upload_f(&mx->kd_f, ax->h_kd));
  FDI_TRY(upload_f(&mx->ko_f, ax->h_ko));
  std::vector<double> wp(n), wm(n), w0(n);
  for (int i = 0; i < n; ++i) {
    const double kp = (i + 1 < n) ? ax->h_ko[i] : 0.0;
    const double km = (i > 0) ? ax->h_ko[i - 1] : 0.0;
    wp[i] = kp / ax->h_m[i];
    wm[i] = km / ax->h_m[i];
    w0[i] = (i == 0 || i == n - 1) ? (ax->h_kd[i] + kp + km) / ax->h_m[i] : 0.0;
  }
  FDI_TRY(upload_df(&mx->wp, wp));
  FDI_TRY(upload_df(&mx->wm, wm));
  FDI_TRY(upload_df(&mx->w0, w0));
  FDI_TRY(upload_df(&mx->m_df, ax->h_m));
  return FDI_OK;
}

}  // namespace

void mixed_free_axis(Axis* ax) {
  MixedAxis* mx = static_cast<MixedAxis*>(ax->mixed);
  if (!mx) return;
  tc_free_matrix(&mx->fwd);
  tc_free_matrix(&mx->bwd);
  void* ptrs[] = {mx->m_f, mx->kd_f, mx->ko_f, mx->wp, mx->wm, mx->w0, mx->m_df, mx->rimg[0], mx->rimg[1]};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  delete mx;
  ax->mixed = nullptr;
}

fdi_status mixed_setup(fdi_plan* p) {
  if (p->prec != FDI_PREC_MIXED_F16) {
    set_error("mixed precision modes other than FDI_PREC_MIXED_F16 are not built");
    return FDI_ERR_UNSUPPORTED;
  }
  if (p->thomas_axis == -1 && p->cyl) {
    set_error("the cylindrical TPF runs on the FP64 path only");
    return FDI_ERR_UNSUPPORTED;
  }
  cudaStream_t s;
  FDI_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  fdi_status st = FDI_OK;
  for (Axis* ax : p->axes) {
    st = setup_axis(p, ax, s);
    if (st != FDI_OK) break;
  }
  cudaError_t e = cudaStreamSynchronize(s);
  cudaStreamDestroy(s);
  if (st != FDI_OK) return st;
  FDI_CUDA_TRY(e);
  FDI_CUDA_TRY(cudaMalloc(&p->d_err, sizeof(int)));
  FDI_CUDA_TRY(cudaMemset(p->d_err, 0, sizeof(int)));
  FDI_CUDA_TRY(cudaMalloc(&p->res_bar, 4 * sizeof(unsigned)));
  FDI_CUDA_TRY(cudaMemset(p->res_bar, 0, 4 * sizeof(unsigned)));
  FDI_CUDA_TRY(cudaStreamCreateWithFlags(&p->cstream, cudaStreamNonBlocking));
  return mixed_alloc_workspace(p);
}

fdi_status mixed_alloc_workspace(fdi_plan* p) {
  size_t szr = 1, szf = 1;
  for (int fi = 0; fi < p->nfields; ++fi) {
    const Field& f = p->fields[fi];
    szr = std::max(szr, (size_t)f.n[2] * f.n[1] * pitch4(f.n[0]));
    szf = std::max(szf, (size_t)f.n[2] * f.n[0] * pitch4(f.n[1]));
  }
  const size_t szw = std::max(szr, szf);  // F1 and F4 take either orientation
  FDI_CUDA_TRY(cudaMalloc(&p->wf[0], szw * sizeof(float)));   // r, reused as F4
  FDI_CUDA_TRY(cudaMalloc(&p->wf[1], szw * sizeof(float)));   // F1
  FDI_CUDA_TRY(cudaMalloc(&p->wf[2], szw * sizeof(float)));   // F2
  FDI_CUDA_TRY(cudaMalloc(&p->wf[3], szw * sizeof(float)));   // Thomas scratch / TPF spectrum F3
  // rows are padded to 4 floats and no pass writes the padding: keep it zero
  // (the TPF z passes read whole padded planes)
  {
    cudaStream_t ms = nullptr;
    FDI_CUDA_TRY(cudaStreamCreateWithFlags(&ms, cudaStreamNonBlocking));
    cudaError_t e = cudaMemsetAsync(p->wf[2], 0, szw * sizeof(float), ms);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->wf[3], 0, szw * sizeof(float), ms);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ms);
    cudaStreamDestroy(ms);
    FDI_CUDA_TRY(e);
  }
  FDI_CUDA_TRY(cudaMalloc(&p->xdf, (size_t)p->Pmax * 3 * sizeof(float)));  // planes H, L, low part of L
  FDI_CUDA_TRY(cudaMalloc(&p->wr1, szr * 2 * sizeof(float)));              // r_1 as (hi, lo) planes
  p->wr1_plane = (long long)szr;
  FDI_CUDA_TRY(cudaMalloc(&p->d_scales, (size_t)(kMaxRefineCap + 2) * kScaleStride * sizeof(float)));
  FDI_CUDA_TRY(cudaMalloc(&p->lam_w, (size_t)10 * kMaxN * sizeof(float2)));
  FDI_CUDA_TRY(cudaMalloc(&p->d_counter, 4 * sizeof(unsigned)));
  FDI_CUDA_TRY(cudaMemset(p->d_counter, 0, 4 * sizeof(unsigned)));
  return FDI_OK;
}

bool resident_eligible(const fdi_plan* p, int field) {
  if (!p || p->prec == FDI_PREC_FP64 || !p->resident || p->cyl || p->thomas_axis != 2) return false;
  if (field < 0 || field >= p->nfields || !p->res_bar) return false;
  const Field& f = p->fields[field];
  if (f.n[0] > kResMaxPlane || f.n[1] > kResMaxPlane) return false;
  for (int d = 0; d < 2; ++d)
    if (!static_cast<const MixedAxis*>(f.ax[d]->mixed)->rimg[0]) return false;
  return true;
}

fdi_status resident_describe(fdi_plan* p, int field, double sigma, double lambda, const double* rhs, double* out,
                             ResJob* job) {
  const Field& f = p->fields[field];
  ResJob& J = *job;
  J = ResJob{};
  J.nx = f.n[0];
  J.ny = f.n[1];
  J.nz = f.n[2];
  J.px = pitch4(J.nx);
  J.cls = (J.nx <= 64 && J.ny <= 64) ? 64 : 128;
  J.singular = (sigma == 0.0 && f.zero_flux_all) ? 1 : 0;
  J.single_pass = p->single_pass ? 1 : 0;
  J.vec = (J.nx % 2 == 0 && (reinterpret_cast<uintptr_t>(rhs) & 15u) == 0 &&
           (reinterpret_cast<uintptr_t>(out) & 15u) == 0) ? 1 : 0;
  J.max_refine = p->max_refine;
  int zc = 0;
  const dim3 rg = resid_grid(J.nx, J.ny, J.nz, &zc);
  J.rgx = (int)rg.x;
  J.rgy = (int)rg.y;
  J.rgz = (int)rg.z;
  J.zchunk = zc;
  if ((long long)J.rgx * J.rgy * J.rgz > p->npartials || J.nz > p->npartials) {
    set_error("grid too large for the reduction buffer");
    return FDI_ERR_INVALID_ARG;
  }
  J.sigma = sigma;
  J.lambda = lambda;
  J.tol = p->tol;
  // FP32 correction residual: error at most about 16 u ||r_1|| (u = 2^-24),
  // kept below tol / 4 of ||b||
  J.fast_limit = p->tol / (4.0 * 16.0 * 5.9604644775390625e-8);
  J.b = rhs;
  J.out = out;
  const MixedAxis* mx = static_cast<const MixedAxis*>(f.ax[0]->mixed);
  const MixedAxis* my = static_cast<const MixedAxis*>(f.ax[1]->mixed);
  const MixedAxis* mz = static_cast<const MixedAxis*>(f.ax[2]->mixed);
  J.kx = (J.nx + 31) / 32;
  J.ky = (J.ny + 31) / 32;
  J.img[0][0] = mx->rimg[0];
  J.img[0][1] = my->rimg[0];
  J.img[1][0] = mx->rimg[1];
  J.img[1][1] = my->rimg[1];
  J.csc[0][0] = mx->fwd.col_scale;
  J.csc[0][1] = my->fwd.col_scale;
  J.csc[1][0] = mx->bwd.col_scale;
  J.csc[1][1] = my->bwd.col_scale;
  J.lamx = f.ax[0]->lam;
  J.lamy = f.ax[1]->lam;
  J.mz = mz->m_f;
  J.kdz = mz->kd_f;
  J.koz = mz->ko_f;
  for (int d = 0; d < 3; ++d) {
    const MixedAxis* m = static_cast<const MixedAxis*>(f.ax[d]->mixed);
    J.w[d][0] = m->wp;
    J.w[d][1] = m->wm;
    J.w[d][2] = m->w0;
    J.m[d] = m->m_df;
  }
  J.lam_w = p->lam_w;
  J.r = p->wf[0];
  J.F = p->wf[2];
  J.cs = p->wf[3];
  J.xh = reinterpret_cast<float*>(p->xdf);
  J.r1 = p->wr1;
  J.r1_plane = p->wr1_plane;
  J.partials = p->partials;
  J.st = p->d_status;
  J.ticket = p->d_counter + 2;
  J.rmax = p->d_scales;
  return FDI_OK;
}

// FP32 Thomas sweep in the configuration of the plan (thomas_tl)
template <bool CYL>
fdi_status launch_thomas32(fdi_plan* p, const Thomas32Args& ta, bool pdl, bool singular, const int* skip,
                           cudaStream_t s) {
  const long long lines = (long long)ta.nx * ta.ny;
  const bool full = ta.nz % kTB == 0;
  if (p->thomas_tl == 2) {
    // two lines per thread, 64 threads (128 lines) per CTA
    const long long pairs = (long long)ta.nx * ((ta.ny + 1) / 2);
    const unsigned g = (unsigned)((pairs + 63) / 64);
    if (full)
      FDI_CUDA_TRY(launch_pdl(pdl, k_thomas2_f32<64, true, CYL>, dim3(g), dim3(64), 0, s, ta, skip));
    else
      FDI_CUDA_TRY(launch_pdl(pdl, k_thomas2_f32<64, false, CYL>, dim3(g), dim3(64), 0, s, ta, skip));
    FDI_LAUNCH_CHECK(p);
    if (singular) {
      // the null line (0, 0) and its pair partner, one line per thread
      Thomas32Args t1 = ta;
      t1.nx = 1;
      t1.ny = std::min(ta.ny, 2);
      if (full)
        k_thomas_f32<64, true, CYL><<<1, 64, 0, s>>>(t1, skip);
      else
        k_thomas_f32<64, false, CYL><<<1, 64, 0, s>>>(t1, skip);
      FDI_LAUNCH_CHECK(p);
    }
    return FDI_OK;
  }
  if (p->thomas_tl == 3) {
    // two lines per thread with the top planes' d' on chip
    static bool attr[2] = {false, false};
    auto kfull = k_thomas2c_f32<true, CYL>;
    auto kpart = k_thomas2c_f32<false, CYL>;
    if (!attr[full ? 1 : 0]) {
      FDI_CUDA_TRY(cudaFuncSetAttribute(full ? kfull : kpart, cudaFuncAttributeMaxDynamicSharedMemorySize, kTopBytes));
      attr[full ? 1 : 0] = true;
    }
    const long long pairs = (long long)ta.nx * ((ta.ny + 1) / 2);
    const unsigned g = (unsigned)((pairs + 63) / 64);
    FDI_CUDA_TRY(launch_pdl(pdl, full ? kfull : kpart, dim3(g), dim3(64), (size_t)kTopBytes, s, ta, skip));
    FDI_LAUNCH_CHECK(p);
    if (singular) {
      Thomas32Args t1 = ta;
      t1.nx = 1;
      t1.ny = std::min(ta.ny, 2);
      if (full)
        k_thomas_f32<64, true, CYL><<<1, 64, 0, s>>>(t1, skip);
      else
        k_thomas_f32<64, false, CYL><<<1, 64, 0, s>>>(t1, skip);
      FDI_LAUNCH_CHECK(p);
    }
    return FDI_OK;
  }
  if (p->thomas_tl == 64) {
    const unsigned g = (unsigned)((lines + 63) / 64);
    if (full)
      FDI_CUDA_TRY(launch_pdl(pdl, k_thomas_f32<64, true, CYL>, dim3(g), dim3(64), 0, s, ta, skip));
    else
      FDI_CUDA_TRY(launch_pdl(pdl, k_thomas_f32<64, false, CYL>, dim3(g), dim3(64), 0, s, ta, skip));
  } else {
    const unsigned g = (unsigned)((lines + 127) / 128);
    if (full)
      FDI_CUDA_TRY(launch_pdl(pdl, k_thomas_f32<128, true, CYL>, dim3(g), dim3(128), 0, s, ta, skip));
    else
      FDI_CUDA_TRY(launch_pdl(pdl, k_thomas_f32<128, false, CYL>, dim3(g), dim3(128), 0, s, ta, skip));
  }
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

fdi_status mixed_field_solve(fdi_plan* p, int field, double sigma, double lambda, const double* rhs, double* out,
                             cudaStream_t s) {
  if (resident_eligible(p, field)) {
    // every pass and refinement round in one cooperative launch
    ResJob job;
    FDI_TRY(resident_describe(p, field, sigma, lambda, rhs, out, &job));
    FDI_KTIMER(p, "resident", s);
    return resident_launch(p, &job, 1, s);
  }
  const Field& f = p->fields[field];
  const int nx = f.n[0], ny = f.n[1], nz = f.n[2];
  const int px = pitch4(nx), py = pitch4(ny);
  const MixedAxis* mx = static_cast<const MixedAxis*>(f.ax[0]->mixed);
  const MixedAxis* my = static_cast<const MixedAxis*>(f.ax[1]->mixed);
  const MixedAxis* mz = static_cast<const MixedAxis*>(f.ax[2]->mixed);
  // (the first pass's reduction resets the solve's status)
  FDI_CUDA_TRY(cudaMemsetAsync(p->d_scales, 0, (size_t)(kMaxRefineCap + 2) * kScaleStride * sizeof(float), s));
  const double* b = rhs;
  if (out == rhs) {
    FDI_CUDA_TRY(cudaMemcpyAsync(p->ws[4], rhs, f.P * sizeof(double), cudaMemcpyDeviceToDevice, s));
    b = p->ws[4];
  }
  const bool singular = sigma == 0.0 && f.zero_flux_all;
  const bool one_pass = p->single_pass;
  float* r = p->wf[0];
  float* F1 = p->wf[1];
  float* F2 = p->wf[2];
  float* CS = p->wf[3];
  float* F4 = p->wf[0];
  // x and y extents that are multiples of 128 allow every pass to write
  // row-major (TMA-stored) outputs: the y and back-x passes then read their
  // inputs with the contraction index strided (MN-major slots)
  const bool mn = nx % 128 == 0 && ny % 128 == 0;
  float* xH = reinterpret_cast<float*>(p->xdf);
  float* xL = xH + f.P;
  float* xLL = xL + f.P;
  float* r1h = p->wr1;
  float* r1l = p->wr1 + p->wr1_plane;
  const int* done = &p->d_status->done;

  int zchunk = kResZChunk;
  const dim3 rgrid = resid_grid(nx, ny, nz, &zchunk);
  const int rblocks = (int)(rgrid.x * rgrid.y * rgrid.z);
  if (rblocks > p->npartials) {
    set_error("grid too large for the reduction buffer");
    return FDI_ERR_INVALID_ARG;
  }
  // flux weights multiplied by lambda for this solve
  {
    FDI_KTIMER(p, "reduce", s);
    k_scale_weights<<<p->cyl ? 10 : 9, 256, 0, s>>>(mx->wp, mx->wm, mx->w0, nx, my->wp, my->wm, my->w0, ny, mz->wp,
                                                    mz->wm, mz->w0, nz, p->cyl_wres_df, nz, split_host(lambda),
                                                    p->lam_w);
    FDI_LAUNCH_CHECK(p);
  }
  ResidArgs ra{};
  ra.nx = nx;
  ra.ny = ny;
  ra.nz = nz;
  for (int d = 0; d < 3; ++d) {
    const MixedAxis* m = static_cast<const MixedAxis*>(f.ax[d]->mixed);
    ra.wp[d] = p->lam_w + (d * 3 + 0) * kMaxN;
    ra.wm[d] = p->lam_w + (d * 3 + 1) * kMaxN;
    ra.w0[d] = p->lam_w + (d * 3 + 2) * kMaxN;
    ra.m[d] = m->m_df;
  }
  ra.wy = p->cyl ? p->lam_w + 9 * kMaxN : nullptr;
  // FP32 correction residual: its error is at most about 16 u ||r_1|| (u =
  // 2^-24; measured near u ||r_1||), kept below tol / 4 of ||b||
  ra.fast_limit = p->tol / (4.0 * 16.0 * 5.9604644775390625e-8);
  ra.sigma = split_host(sigma);
  ra.lambda = split_host(lambda);
  ra.sig_mode = sigma == 0.0 ? 0 : (sigma == 1.0 ? 1 : 2);
  ra.b = b;
  ra.r = r;
  ra.r_pitch = px;
  ra.zchunk = zchunk;
  ra.st = p->d_status;
  ra.partials = p->partials;

  // r_0 = b (and the volume-weighted mean of b for the singular problem)
  const int iblocks = 152 * 8;
  {
    FDI_KTIMER(p, "residual_df_init", s);
    ResidArgs a0 = ra;
    a0.xh = nullptr;
    a0.xl = nullptr;
    a0.out = nullptr;
    a0.sub_mean = 0;
    a0.want_mean = singular ? 1 : 0;
    a0.rmax = p->d_scales + 0;
    a0.fin = FinishArgs{p->d_counter, p->partials, p->d_status, p->tol, 0, singular ? 1 : 0};
    if (px == nx && !singular && (reinterpret_cast<uintptr_t>(b) & 15u) == 0)
      FDI_CUDA_TRY(launch_pdl(true, k_init_rhs_flat, dim3(iblocks), dim3(256), 0, s, a0, f.P));
    else  // one warp per x-line: no more blocks than lines / 8
      FDI_CUDA_TRY(launch_pdl(true, k_init_rhs, dim3(std::min(iblocks, (ny * nz + 7) / 8)), dim3(256), 0, s, a0));
    FDI_LAUNCH_CHECK(p);
  }

  // one refinement round (round 0: the first solve) enqueued on stream s;
  // next_round: graph condition the round's residual check sets
  auto enqueue_round = [&](int round, cudaStream_t s, cudaGraphConditionalHandle next_round) -> fdi_status {
    const bool pdl = p->pdl && round < 2;  // later rounds may run inside conditional graph bodies
    const int* skip = round == 0 ? nullptr : done;
    float* sc = p->d_scales + kScaleStride * round;
    float* sc_next = p->d_scales + kScaleStride * (round + 1);
    // forward x: r [z][y][x] -> F1 [z][i][y] (round 1 reads r_1 from its own planes)
    TcArgs t{};
    t.pdl = pdl ? 1 : 0;
    t.skip = skip;
    t.err = p->d_err;
    t.in = round == 1 ? r1h : r;
    t.R = (long long)nz * ny;
    t.K = nx;
    t.in_pitch = px;
    t.scale_in = sc + 0;
    t.mode = TC_OUT_F32;
    t.n_out = nx;
    t.out_f32 = F1;
    if (mn) {
      // F1 [z][y][i] (row-major, TMA stores)
      t.S = t.R;
      t.slab_stride = 0;
      t.row_stride = px;
      t.col_stride = 1;
    } else {
      // F1 [z][i][y] (transposed)
      t.S = ny;
      t.slab_stride = (long long)nx * py;
      t.row_stride = 1;
      t.col_stride = py;
    }
    t.scale_out = sc + 1;
    FDI_TRY(launch_tc_transform(p, mx->fwd, t, "transform_xf_tc", s));
    // forward y: F1 -> F2 [z][i][j]; rows (z, i), contraction over y
    t.in = F1;
    t.R = (long long)nz * nx;
    t.K = ny;
    t.in_pitch = mn ? px : py;
    t.a_mn = mn ? 1 : 0;          // F1 [z][y][i]: i contiguous
    t.a_mslab = nx;
    t.a_rows = (long long)nz * ny;
    t.scale_in = sc + 1;
    t.n_out = ny;
    t.out_f32 = F2;
    t.S = t.R;
    t.slab_stride = 0;
    t.row_stride = py;
    t.col_stride = 1;
    const bool tpf = p->thomas_axis == -1;
    t.scale_out = tpf ? sc + 4 : nullptr;  // TPF: the z transform needs the scale of F2
    FDI_TRY(launch_tc_transform(p, my->fwd, t, "transform_yf_tc", s));
    if (tpf) {
      // TPF (Eq. 29): z transform, spectral divide, back z transform.  F2
      // [z][i][j] is read with the contraction index z strided: the padded
      // plane (nx * py values) is one MN-major slab of R = nx * py rows, and
      // the transforms write [z'][i][j] back in the same layout
      const int plane = nx * py;
      TcArgs tz{};
      tz.pdl = t.pdl;
      tz.skip = skip;
      tz.err = p->d_err;
      tz.in = F2;
      tz.R = plane;
      tz.K = nz;
      tz.in_pitch = plane;
      tz.a_mn = 1;
      tz.a_mslab = plane;
      tz.a_rows = nz;
      tz.scale_in = sc + 4;
      tz.mode = TC_OUT_F32;
      tz.n_out = nz;
      tz.out_f32 = CS;
      tz.S = plane;
      tz.slab_stride = 0;
      tz.row_stride = 1;
      tz.col_stride = plane;
      tz.scale_out = nullptr;  // the divide measures its own output
      FDI_TRY(launch_tc_transform(p, mz->fwd, tz, "transform_zf_tc", s));
      {
        FDI_KTIMER(p, "divide_f32", s);
        const long long rows = (long long)nz * nx;
        FDI_CUDA_TRY(launch_pdl(pdl, k_divide_tpf, dim3((unsigned)std::min<long long>((rows + 7) / 8, 152 * 8)),
                                dim3(256), 0, s, CS, nx, ny, py, nz, (const double*)f.ax[0]->lam,
                                (const double*)f.ax[1]->lam, (const double*)f.ax[2]->lam, sigma, lambda,
                                singular ? 1 : 0, sc + 5, skip));
        FDI_LAUNCH_CHECK(p);
      }
      tz.in = CS;
      tz.scale_in = sc + 5;
      tz.out_f32 = F2;
      tz.scale_out = sc + 2;
      FDI_TRY(launch_tc_transform(p, mz->bwd, tz, "transform_zb_tc", s));
    } else {
      // Thomas along z, in place on F2
      FDI_KTIMER(p, "thomas_z_f32", s);
      Thomas32Args ta;
      ta.f = F2;
      ta.cs = CS;
      ta.nx = nx;
      ta.ny = ny;
      ta.nz = nz;
      ta.pitch = py;
      ta.plane = (long long)nx * py;
      ta.lamx = f.ax[0]->lam;
      ta.lamy = f.ax[1]->lam;
      ta.mz = mz->m_f;
      ta.kdz = mz->kd_f;
      ta.koz = mz->ko_f;
      ta.sigma = sigma;
      ta.lambda = lambda;
      ta.singular_possible = singular ? 1 : 0;
      ta.fmax = sc + 2;
      ta.wy = p->cyl ? p->cyl_wy_f : nullptr;
      if (p->thomas_tl == 4 && p->tf && !singular)
        FDI_TRY(launch_thomas_cached_f32(p, f, sigma, lambda, field, F2, py, (long long)nx * py, sc + 2, skip, s));
      else if (p->cyl)
        FDI_TRY(launch_thomas32<true>(p, ta, pdl, singular, skip, s));
      else
        FDI_TRY(launch_thomas32<false>(p, ta, pdl, singular, skip, s));
    }
    // back y: F2 [z][i][j] -> F4
    t.in = F2;
    t.R = (long long)nz * nx;
    t.K = ny;
    t.in_pitch = py;
    t.a_mn = 0;
    t.scale_in = sc + 2;
    t.n_out = ny;
    t.out_f32 = F4;
    if (mn) {
      // F4 [z][i][y] (row-major, TMA stores)
      t.S = t.R;
      t.slab_stride = 0;
      t.row_stride = py;
      t.col_stride = 1;
    } else {
      // F4 [z][y][i] (transposed)
      t.S = nx;
      t.slab_stride = (long long)ny * px;
      t.row_stride = 1;
      t.col_stride = px;
    }
    t.scale_out = sc + 3;
    FDI_TRY(launch_tc_transform(p, my->bwd, t, "transform_yb_tc", s));
    // back x: F4 -> H (first solve), L (first correction) or L += (later ones), [z][y][x];
    // rows (z, y), contraction over i
    t.in = F4;
    t.R = (long long)nz * ny;
    t.K = nx;
    t.in_pitch = mn ? py : px;
    t.a_mn = mn ? 1 : 0;          // F4 [z][i][y]: y contiguous
    t.a_mslab = ny;
    t.a_rows = (long long)nz * nx;
    t.scale_in = sc + 3;
    t.mode = round <= 1 ? TC_OUT_F32 : TC_OUT_DF_ADD;
    t.n_out = nx;
    t.out_f32 = round == 0 ? xH : xL;
    t.out_lo = xLL;
    t.lo_valid = round >= 3 ? 1 : 0;
    t.S = t.R;
    t.slab_stride = 0;
    t.row_stride = nx;
    t.col_stride = 1;
    t.scale_out = nullptr;
    FDI_TRY(launch_tc_transform(p, mx->bwd, t,
                                round == 0 ? "transform_xb_set_tc" : (round == 1 ? "transform_xb_corr_tc" : "transform_xb_add_tc"),
                                s));
    // residual and convergence check: r_1 = b - A H after the first solve,
    // r = r_1 - A L after each correction (which also writes the FP64 solution)
    if (!one_pass) {
      FDI_KTIMER(p, round == 0 ? "residual_df" : "residual_corr", s);
      ResidArgs ak = ra;
      ak.xh = xH;
      ak.xl = xL;
      ak.xll = xLL;
      ak.r1 = r1h;
      ak.r1_lo = r1l;
      ak.r = round == 0 ? r1h : r;
      ak.r_lo = r1l;
      ak.out = out;
      ak.rmax = sc_next + 0;
      ak.fin = FinishArgs{p->d_counter, p->partials, p->d_status, p->tol, round == 0 ? 1 : 2, singular ? 1 : 0,
                          next_round};
      const bool write_out = !singular && round > 0;
      const bool vec = nx % 2 == 0 && (reinterpret_cast<uintptr_t>(b) & 15u) == 0 &&
                       (reinterpret_cast<uintptr_t>(out) & 15u) == 0;
      ResidKernel kern = resid_kernel(ra.sig_mode, round == 0 ? 0 : 1, round >= 2, singular, write_out, p->cyl, vec);
      FDI_CUDA_TRY(launch_pdl(pdl, kern, rgrid, dim3(kResTX, kResTY), 0, s, ak, skip));
      FDI_LAUNCH_CHECK(p);
    }
      return FDI_OK;
  };
  // Eagerly, every round is enqueued and returns at once after convergence.
  // In a captured solve, round r >= 2 sits in a conditional graph node placed
  // (nested) in round r-1's graph, whose residual check sets the condition, so
  // a converged solve launches nothing more.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaGraph_t cgraph = nullptr;
  bool conditional = false;
  if (!one_pass && p->max_refine >= 2 && p->cstream &&
      cudaStreamGetCaptureInfo(s, &cap, nullptr, &cgraph, nullptr, nullptr, nullptr) == cudaSuccess &&
      cap == cudaStreamCaptureStatusActive && cgraph) {
    // add an IF node after the current capture point of `st` (capturing into
    // `g`); returns its body graph
    auto add_if = [&](cudaStream_t st, cudaGraph_t g, cudaGraphConditionalHandle h, cudaGraph_t* body) -> fdi_status {
      const cudaGraphNode_t* deps = nullptr;
      size_t ndeps = 0;
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      cudaGraph_t gg = nullptr;
      FDI_CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &gg, &deps, nullptr, &ndeps));
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeIf;
      cp.conditional.size = 1;
      cudaGraphNode_t node = nullptr;
      FDI_CUDA_TRY(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp));
      FDI_CUDA_TRY(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
      *body = cp.conditional.phGraph_out[0];
      return FDI_OK;
    };
    conditional = true;
    cudaGraphConditionalHandle h = 0;
    FDI_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, cgraph, 0, cudaGraphCondAssignDefault));
    FDI_TRY(enqueue_round(0, s, 0));
    FDI_TRY(enqueue_round(1, s, h));
    cudaGraph_t body = nullptr;
    FDI_TRY(add_if(s, cgraph, h, &body));
    for (int r = 2; r <= p->max_refine; ++r) {
      cudaGraphConditionalHandle hn = 0;
      if (r < p->max_refine) FDI_CUDA_TRY(cudaGraphConditionalHandleCreate(&hn, body, 0, cudaGraphCondAssignDefault));
      FDI_CUDA_TRY(cudaStreamBeginCaptureToGraph(p->cstream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
      fdi_status st = enqueue_round(r, p->cstream, hn);
      cudaGraph_t next_body = nullptr;
      if (st == FDI_OK && hn) st = add_if(p->cstream, body, hn, &next_body);
      cudaGraph_t done_graph = nullptr;
      const cudaError_t e = cudaStreamEndCapture(p->cstream, &done_graph);
      FDI_TRY(st);
      FDI_CUDA_TRY(e);
      body = next_body;
    }
  } else {
    for (int round = 0; round <= (one_pass ? 0 : p->max_refine); ++round) FDI_TRY(enqueue_round(round, s, 0));
  }
  {
    // FP64 output when the loop stopped before its last round (and, for the
    // zero-flux Laplace problem, minus the volume-weighted mean: the FP32 sweep
    // projects the null line only to single precision, and the constant is
    // outside the range of A, so shifting it leaves the residual)
    // after a conditional node the launch is an ordinary one: a programmatic
    // edge needs a kernel upstream, and this pass reads what the node's body
    // writes
    FDI_KTIMER(p, "finalize_out", s);
    // (single pass: out = H, no refinement step and no mean removal)
    FDI_CUDA_TRY(launch_pdl(!conditional, k_finalize_out, dim3(kBlocks), dim3(kThreads), 0, s, (const float*)xH,
                            (const float*)xL, (const float*)xLL, out, f.P, (const DevStatus*)p->d_status,
                            one_pass ? 1 : p->max_refine, (singular && !one_pass) ? 1 : 0));
    FDI_LAUNCH_CHECK(p);
  }
  return FDI_OK;
}


}  // namespace fdi

extern "C" fdi_status fdi_apply_transform(fdi_plan* plan, fdi_field field, int d, int inverse, const float* in,
                                          float* out, long long rows, fdi_stream_t stream) {
  using namespace fdi;
  if (!plan || !in || !out || rows < 0 || d < 0 || d > 2 || (int)field < 0 || (int)field >= plan->nfields)
    return FDI_ERR_INVALID_ARG;
  if (plan->prec != FDI_PREC_MIXED_F16) {
    set_error("fdi_apply_transform needs a FDI_PREC_MIXED_F16 plan");
    return FDI_ERR_UNSUPPORTED;
  }
  if (rows == 0) return FDI_OK;
  int di = d;  // internal axis holding external direction d
  for (int q = 0; q < 3; ++q)
    if (plan->perm[q] == d) di = q;
  const Axis* ax = plan->fields[(int)field].ax[di];
  const MixedAxis* m = static_cast<const MixedAxis*>(ax->mixed);
  const int n = ax->n, pitch = pitch4(n);
  cudaStream_t s = (cudaStream_t)stream;
  // input scale: max |in| reduced on the device into the first scale slot
  FDI_CUDA_TRY(cudaMemsetAsync(plan->d_scales, 0, 4 * sizeof(float), s));
  k_absmax<<<152 * 4, 256, 0, s>>>(in, rows, n, pitch, plan->d_scales);
  FDI_LAUNCH_CHECK(plan);
  TcArgs t{};
  t.in = in;
  t.R = rows;
  t.K = n;
  t.in_pitch = pitch;
  t.scale_in = plan->d_scales;
  t.mode = TC_OUT_F32;
  t.n_out = n;
  t.out_f32 = out;
  t.S = rows;
  t.row_stride = pitch;
  t.col_stride = 1;
  t.err = plan->d_err;
  return launch_tc_transform(plan, inverse ? m->fwd : m->bwd, t, inverse ? "transform_fwd_tc" : "transform_bwd_tc", s);
}

extern "C" fdi_status fdi_plan_set_wait_limit(fdi_plan* plan, long long cycles) {
  if (!plan || cycles < 0) return FDI_ERR_INVALID_ARG;
  plan->wait_cycles = cycles;
  fdi::invalidate_graph(plan);  // the limit is a kernel argument of captured launches
  if (plan->d_err) {
    // nothing of this plan may still run while its flag is cleared
    FDI_CUDA_TRY(cudaDeviceSynchronize());
    FDI_CUDA_TRY(cudaMemset(plan->d_err, 0, sizeof(int)));
  }
  return FDI_OK;
}

extern "C" fdi_status fdi_plan_set_resident(fdi_plan* plan, int enable) {
  if (!plan || (enable != 0 && enable != 1)) return FDI_ERR_INVALID_ARG;
  plan->resident = enable;
  fdi::invalidate_graph(plan);  // captured solves took the other route
  return FDI_OK;
}
