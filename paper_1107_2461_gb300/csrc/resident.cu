// Resident small-grid solve: one cooperative launch runs every pass of the
// mixed-precision TPT solve (Sec. 3, end: E_x^{-1}, E_y^{-1}, Thomas along z,
// E_y, E_x) and all of its refinement rounds, for one or several independent
// field solves at once (the three velocity components of a Stokes step,
// Sec. 2; a batch of uneven grids).  The CTAs meet at a grid barrier between
// passes instead of at a kernel boundary, so a solve costs one launch.
//
// A field qualifies when its x and y extents are at most 128.  A z-plane then
// fits in shared memory and one CTA applies both plane transforms to it,
// G = E_y^{-1} P E_x^{-T}, as two FP32 products on the CUDA cores.  At these
// sizes a pass moves a few MB: it is bound by latency (launch, barrier,
// dependent steps of the sweep), not by HBM or the tensor pipe, and plain FP32
// needs none of the split-precision scaling of the tensor-core passes.
//
// Passes of one refinement round, each over every active solve (units handed
// to the CTAs round-robin):
//   F  forward plane transforms, one unit per (solve, z-plane); round 0 reads
//      b (FP64) and also reduces ||b||^2 (and the volume-weighted mean of b
//      for the zero-flux Laplace problem), the first residual r_1, later
//      rounds the correction residual
//   T  Thomas sweep along z, one unit per (solve, tile of (x-mode, y-mode) lines)
//   B  back plane transforms: H (round 0), L (round 1), (L, L_lo) += (later)
//   R  the double-float residual of the pass-by-pass solve (same body), one
//      unit per (solve, residual block); the solve's last unit runs the
//      fixed-order reduction and the convergence check
// A solve's arithmetic does not depend on which CTA runs a unit, on the grid
// size or on the other solves of the launch: results are bitwise those of the
// solve launched alone.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "df.cuh"
#include "fdi_internal.h"
#include "resid.cuh"
#include "resident.h"
#include "tc_common.cuh"

namespace fdi {

namespace {

constexpr int kRT = 256;        // threads per CTA: 32 x 8 (residual), 16 x 16 (plane products)

struct ResLaunch {
  int njobs;
  int max_rounds;      // largest max_refine over the solves (0: single pass only)
  unsigned* bar;       // grid barrier: arrivals, generation, abort flag, exits
  int* err;            // wait-limit flag of the launching plan
  long long wait;      // barrier and tensor-memory wait limit, cycles
  int cls;             // largest plane class of the solves: the shared-memory regions
  ResJob job[kResMaxJobs];
};
static_assert(sizeof(ResLaunch) <= 32000, "kernel parameter block too large");

// ---- grid barrier (cooperative launch: every CTA is resident) ----

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// All CTAs arrive (acquire-release add on the arrival count); the last one
// resets the count and publishes the next generation (release), the others
// wait for it (acquire): what a CTA wrote before the barrier is visible to
// every CTA after it.  Bounded: a wait that runs out raises the abort flag and
// the plan's error flag, and every CTA then leaves at its next barrier.
__device__ bool grid_barrier(const ResLaunch& L, int tid, int* s_ok) {
  __syncthreads();
  if (tid == 0) {
    unsigned* bar = L.bar;
    int ok = ld_acquire(bar + 2) == 0u;
    if (ok) {
      const unsigned g = ld_acquire(bar + 1);
      if (atom_add_acq_rel(bar, 1u) == gridDim.x - 1) {
        bar[0] = 0u;
        st_release(bar + 1, g + 1u);
      } else {
        const long long t0 = clock64();
        for (unsigned it = 1; ld_acquire(bar + 1) == g; ++it) {
          if ((it & 15u) == 0u) {
            if (ld_acquire(bar + 2) != 0u) {
              ok = 0;
              break;
            }
            if (clock64() - t0 > L.wait) {
              atomicExch(bar + 2, 1u);
              atomicExch(L.err, 8);
              ok = 0;
              break;
            }
          }
        }
      }
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Last CTA out re-arms the barrier and the solves' tickets for the next
// launch (also after an abort, when counts may be left over).  No wait.
__device__ void grid_exit(const ResLaunch& L, int tid) {
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(L.bar + 3, 1u) == gridDim.x - 1) {
      for (int q = 0; q < L.njobs; ++q) *L.job[q].ticket = 0u;
      L.bar[0] = 0u;
      L.bar[2] = 0u;
      __threadfence();
      L.bar[3] = 0u;
    }
  }
}

// ---- units of a pass ----

enum { U_PLANE = 0, U_LINES = 1, U_RESID = 2, U_OUT = 3, U_LINES0 = 4 };
constexpr int kOutChunk = kRT * 8;  // points per output unit

__device__ __forceinline__ int unit_count(const ResJob& J, int kind) {
  switch (kind) {
    case U_PLANE: return J.nz;
    case U_LINES: return (J.ny * J.px + J.lt - 1) / J.lt;
    case U_LINES0: return (J.ny * J.px + J.lt - 1) / J.lt + 1;  // and the first pass's reduction
    case U_RESID: return J.rgx * J.rgy * J.rgz;
    default: return (int)(((long long)J.nx * J.ny * J.nz + kOutChunk - 1) / kOutChunk);
  }
}

// unit u of the pass (active solves in launch order) -> (solve, local unit)
__device__ __forceinline__ bool unit_of(const ResLaunch& L, const unsigned char* active, int kind, int u, int* q,
                                        int* loc) {
  for (int j = 0; j < L.njobs; ++j) {
    if (!active[j]) continue;
    const int c = unit_count(L.job[j], kind);
    if (u < c) {
      *q = j;
      *loc = u;
      return true;
    }
    u -= c;
  }
  return false;
}

__device__ __forceinline__ int units_total(const ResLaunch& L, const unsigned char* active, int kind) {
  int t = 0;
  for (int j = 0; j < L.njobs; ++j)
    if (active[j]) t += unit_count(L.job[j], kind);
  return t;
}

// ---- staging ----

// 16-byte asynchronous copy global -> shared (L2 only), and the wait for all
// of a thread's copies
__device__ __forceinline__ void cp16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// issue the copy of rows j < ny of an FP32 plane (row pitch px, a multiple of
// 4) into the tile, zero elsewhere (the caller waits)
__device__ __forceinline__ void stage_plane(float* dst, int sp, int cls, const float* src, int ny, int px, int tid) {
  const int g = cls / 4;
  for (int e = tid; e < cls * g; e += kRT) {
    const int j = e / g, c = (e % g) * 4;
    if (j < ny && c < px)
      cp16(dst + j * sp + c, src + (long long)j * px + c);
    else
      *reinterpret_cast<float4*>(dst + j * sp + c) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// ---- reductions shared by the passes ----

// the unit's contribution is in; true (CTA-uniform) for the solve's last unit
// of the pass, which then sees every other unit's partials
__device__ __forceinline__ bool last_unit(const ResJob& J, int count, int tid, unsigned* s_last) {
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    *s_last = atomicAdd(J.ticket, 1u) == (unsigned)(count - 1) ? 1u : 0u;
  }
  __syncthreads();
  const bool last = *s_last != 0u;
  if (last) __threadfence();
  return last;
}

// ---- plane transforms on the tensor cores ----
//
// One unit applies both plane transforms to z-plane k of a solve, y first:
//   forward  D1[i][m] = sum_j P[j][i] E_y^{-1}[m][j],  G[m][k'] = sum_i D1[i][m] E_x^{-1}[k'][i]
//   back     D1[k'][j] = sum_m S[m][k'] E_y[j][m],     X[j][i] = sum_k' D1[k'][j] E_x[i][k']
// (Eq. 25 along y, then along x).  Each product is a tcgen05 MMA (kind::f16,
// M = 128, N = 32 k, K in chunks of 32) with both operands split into fp16 hi
// and lo parts and A_hi B_hi + A_hi B_lo + A_lo B_hi accumulated in FP32 in
// tensor memory, as in the pass-by-pass transforms.  The plane's columns are
// the rows of the first left operand (written transposed, K-major, while it
// is split); the first result's columns are the rows of the second (written
// transposed from tensor memory).  Each left operand is scaled by the power
// of two that maps its largest magnitude into [2^14, 2^15); the matrices'
// rows carry their own scales, undone per output column.
//
// Shared memory (1024-byte aligned regions): S, the FP32 plane (pitch
// cls + 4), then the second matrix image; A, the left operand (per K chunk
// the hi then the lo 128 x 64-byte rows); B, the first matrix image.

constexpr int kAHalf = 128 * 64;      // one half (hi or lo) of a K chunk of the left operand
constexpr int kAChunk = 2 * kAHalf;

__host__ __device__ constexpr int res_s_bytes(int cls) { return ((cls * (cls + 4) * 4 + 1023) / 1024) * 1024; }
__host__ __device__ constexpr int res_a_bytes(int cls) { return (cls / 32) * kAChunk; }
__host__ __device__ constexpr int res_b_bytes(int cls) { return (cls / 32) * 2 * cls * 64; }

struct PlaneSmem {
  uint8_t* S;
  uint8_t* A;
  uint8_t* B;
};

// power of two mapping mx into [2^14, 2^15) (1 for zero or non-finite mx)
__device__ __forceinline__ float res_scale(float mx) {
  const uint32_t b = __float_as_uint(mx);
  const int e = (int)((b >> 23) & 0xff);
  if (e == 0 || e == 255) return 1.0f;
  int se = 127 + 14 - (e - 127);
  se = se < 1 ? 1 : (se > 254 ? 254 : se);
  return __uint_as_float((uint32_t)se << 23);
}

// maximum over the CTA (every thread gets it)
__device__ __forceinline__ float block_max(float v, float* redf, int tid) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((tid & 31) == 0) redf[tid / 32] = v;
  __syncthreads();
  float m = redf[0];
#pragma unroll
  for (int w = 1; w < kRT / 32; ++w) m = fmaxf(m, redf[w]);
  __syncthreads();
  return m;
}

// D (tensor memory) = A B^T over nk K chunks, three split products each
__device__ __forceinline__ void issue_split_gemm(uint32_t d, uint32_t a, uint32_t b, int nk, int npad) {
  const uint32_t idesc = tc::idesc_f16_f32(128, npad);
  for (int kc = 0; kc < nk; ++kc) {
    const uint32_t ahi = a + kc * kAChunk, alo = ahi + kAHalf;
    const uint32_t bhi = b + kc * (2 * npad * 64), blo = bhi + npad * 64;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
      const uint32_t off = kk * 32;
      const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
      tc::mma_f16(d, tc::sdesc_k_sw64(ahi + off), tc::sdesc_k_sw64(bhi + off), idesc, acc);
      tc::mma_f16(d, tc::sdesc_k_sw64(ahi + off), tc::sdesc_k_sw64(blo + off), idesc, 1u);
      tc::mma_f16(d, tc::sdesc_k_sw64(alo + off), tc::sdesc_k_sw64(bhi + off), idesc, 1u);
    }
  }
}

// one 32-column segment (group g) of row `row` of the spectral plane k (the
// padded row: zero past nx)
__device__ __forceinline__ void store_row(const ResJob& J, int k, int row, int g, const uint32_t (&r)[32],
                                          const float* cs2, float isb) {
  float* Fr = J.F + ((long long)k * J.ny + row) * J.px + 32 * g;
#pragma unroll
  for (int c = 0; c < 32; c += 4)
    if (32 * g + c < J.px)
      *reinterpret_cast<float4*>(Fr + c) =
          make_float4(__uint_as_float(r[c]) * cs2[32 * g + c] * isb, __uint_as_float(r[c + 1]) * cs2[32 * g + c + 1] * isb,
                      __uint_as_float(r[c + 2]) * cs2[32 * g + c + 2] * isb,
                      __uint_as_float(r[c + 3]) * cs2[32 * g + c + 3] * isb);
}

// One unit: plane k of solve J, forward (dir 0: b or a residual -> spectral
// plane) or back (dir 1: spectral plane -> H, L or the FP64 output).  False
// when a tensor-memory wait ran out (the caller aborts the launch).
__device__ bool unit_plane(const ResJob& J, int dir, int round, int k, const PlaneSmem& ps, uint32_t tbase,
                           uint64_t* mbar, uint32_t& mph, int tid, float* redf, double* red, unsigned* s_last,
                           volatile int* s_abort, long long wait) {
  const int nx = J.nx, ny = J.ny, cls = J.cls, sp = cls + 4;
  const int kx = J.kx, ky = J.ky, nxp = 32 * kx, nyp = 32 * ky;
  const int warp = tid / 32, lane = tid % 32, q = warp % 4, colh = warp / 4;
  float* S = reinterpret_cast<float*>(ps.S);
  // 1. the first matrix image and the plane
  {
    const uint8_t* src = J.img[dir][1];
    const int bytes = ky * 2 * nyp * 64;
    for (int e = tid * 16; e < bytes; e += kRT * 16) cp16(ps.B + e, src + e);
  }
  const int g4 = cls / 4;
  float sbb = 0.f;
  df::F2 svb = df::make(0.f, 0.f), sv = df::make(0.f, 0.f);
  const bool first = dir == 0 && round == 0;
  const bool mean = first && J.singular;
  if (first) {
    // r_0 = b rounded to FP32; ||b||^2 and the volume-weighted sums of the plane
    df::F2 vzk = df::make(0.f, 0.f);
    if (mean) vzk = df::make(J.m[2][k].x, J.m[2][k].y);
    const double* bk = J.b + (long long)k * ny * nx;
    for (int e0 = tid; e0 < cls * g4; e0 += 4 * kRT) {
      double v[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * kRT, j = e / g4, c = (e % g4) * 4;
#pragma unroll
        for (int w = 0; w < 4; ++w)
          v[u][w] = (e < cls * g4 && j < ny && c + w < nx) ? bk[(long long)j * nx + c + w] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + u * kRT, j = e / g4, c = (e % g4) * 4;
        if (e >= cls * g4) break;
        float w4[4] = {0.f, 0.f, 0.f, 0.f};
        if (j < ny) {
          df::F2 vjk = df::make(0.f, 0.f);
          if (mean) vjk = df::mul(df::make(J.m[1][j].x, J.m[1][j].y), vzk);
#pragma unroll
          for (int w = 0; w < 4; ++w)
            if (c + w < nx) {
              const df::F2 bb = df::from_f64(v[u][w]);
              w4[w] = bb.hi + bb.lo;
              sbb = fmaf(w4[w], w4[w], sbb);
              if (mean) {
                const df::F2 V = df::mul(vjk, df::make(J.m[0][c + w].x, J.m[0][c + w].y));
                svb = df::add(svb, df::mul(V, bb));
                sv = df::add(sv, V);
              }
            }
        }
        *reinterpret_cast<float4*>(S + j * sp + c) = make_float4(w4[0], w4[1], w4[2], w4[3]);
      }
    }
  } else if (dir == 0) {
    stage_plane(S, sp, cls, (round == 1 ? J.r1 : J.r) + (long long)k * ny * J.px, ny, J.px, tid);
  } else {
    stage_plane(S, sp, cls, J.F + (long long)k * ny * J.px, ny, J.px, tid);
  }
  cp_wait_all();
  tc::fence_proxy_async_smem();  // the image, for the tensor cores
  __syncthreads();
  if (dir == 0 && round != 0 && J.px > nx) {
    // the residual planes' row padding holds no value: zero it in the tile
    const int pad = J.px - nx;
    for (int e = tid; e < ny * pad; e += kRT) S[(e / pad) * sp + nx + e % pad] = 0.f;
    __syncthreads();
  }
  // 2. left operand 1: row = plane column (< 128), K = plane row (< nyp)
  float mx = 0.f;
  for (int e = tid; e < ny * g4; e += kRT) {
    const float4 v = *reinterpret_cast<const float4*>(S + (e / g4) * sp + (e % g4) * 4);
    mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
  const float sa = res_scale(block_max(mx, redf, tid));
  for (int t = tid; t < 128 * 4 * ky; t += kRT) {
    const int row = t % 128, oct = t / 128;
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      const int j = 8 * oct + e;
      const float x0 = (row < cls && j < cls) ? S[j * sp + row] * sa : 0.f;
      const float x1 = (row < cls && j + 1 < cls) ? S[(j + 1) * sp + row] * sa : 0.f;
      const __half2 h = __floats2half2_rn(x0, x1);
      const float2 hf = __half22float2(h);
      const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
      hw[e / 2] = *reinterpret_cast<const uint32_t*>(&h);
      lw[e / 2] = *reinterpret_cast<const uint32_t*>(&l);
    }
    const uint32_t off = (uint32_t)((oct / 4) * kAChunk) + tc::sw64_offset(row, (oct % 4) * 8);
    *reinterpret_cast<uint4*>(ps.A + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(ps.A + off + kAHalf) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
  __syncthreads();  // the plane is consumed: its space takes the second image
  {
    const uint8_t* src = J.img[dir][0];
    const int bytes = kx * 2 * nxp * 64;
    for (int e = tid * 16; e < bytes; e += kRT * 16) cp16(ps.S + e, src + e);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  tc::fence_proxy_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (tid == 0) {
    issue_split_gemm(tbase, tc::smem_u32(ps.A), tc::smem_u32(ps.B), ky, nyp);
    tc::mma_commit(mbar);
    *s_abort = tc::mbar_wait(mbar, mph, s_abort, wait) ? 0 : 1;
  }
  __syncthreads();
  if (*s_abort) return false;
  mph ^= 1u;
  tc::tc_fence_after();
  // 3. D1: lanes = plane columns, columns = y outputs (< nyp)
  const float* cs1 = J.csc[dir][1];
  const float isa = 1.0f / sa;
  float m2 = 0.f;
  uint32_t ra[32];  // this warp's first column group of D1, kept for the conversion
  if (colh < ky) {
    tc::tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * colh), ra);
    tc::tmem_ld_wait();
#pragma unroll
    for (int c = 0; c < 32; ++c) m2 = fmaxf(m2, fabsf(__uint_as_float(ra[c]) * cs1[32 * colh + c] * isa));
  }
  for (int g = colh + 2; g < ky; g += 2) {
    uint32_t r[32];
    tc::tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * g), r);
    tc::tmem_ld_wait();
#pragma unroll
    for (int c = 0; c < 32; ++c) m2 = fmaxf(m2, fabsf(__uint_as_float(r[c]) * cs1[32 * g + c] * isa));
  }
  const float sb = res_scale(block_max(m2, redf, tid));
  // left operand 2: row = D1 column, K = D1 lane (chunk q, position lane);
  // lanes past the x extent's chunks carry zeros and are not needed
  auto put_a2 = [&](int g, const uint32_t (&r)[32]) {
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      const float x = __uint_as_float(r[c]) * cs1[32 * g + c] * isa * sb;
      const __half h = __float2half_rn(x);
      const __half l = __float2half_rn(x - __half2float(h));
      const uint32_t off = (uint32_t)(q * kAChunk) + tc::sw64_offset(32 * g + c, lane);
      *reinterpret_cast<__half*>(ps.A + off) = h;
      *reinterpret_cast<__half*>(ps.A + off + kAHalf) = l;
    }
  };
  if (q < kx) {
    if (colh < ky) put_a2(colh, ra);
    for (int g = colh + 2; g < ky; g += 2) {
      uint32_t r[32];
      tc::tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * g), r);
      tc::tmem_ld_wait();
      put_a2(g, r);
    }
  }
  cp_wait_all();                 // the second image
  tc::fence_proxy_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (tid == 0) {
    issue_split_gemm(tbase, tc::smem_u32(ps.A), tc::smem_u32(ps.S), kx, nxp);
    tc::mma_commit(mbar);
    *s_abort = tc::mbar_wait(mbar, mph, s_abort, wait) ? 0 : 1;
  }
  __syncthreads();
  if (*s_abort) return false;
  mph ^= 1u;
  tc::tc_fence_after();
  // 4. D2: lanes = y (output rows), columns = x outputs (< nxp)
  const float* cs2 = J.csc[dir][0];
  const float isb = 1.0f / sb;
  const int row = 32 * q + lane;
  const long long P = (long long)nx * ny * J.nz;
  for (int g = colh; g < kx; g += 2) {
    uint32_t r[32];
    tc::tmem_ld32(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * g), r);
    tc::tmem_ld_wait();
    if (row < ny) {
      if (dir == 0) {
        store_row(J, k, row, g, r, cs2, isb);
      } else {
        // into the tile (its image was consumed by the product), rows of the plane
#pragma unroll
        for (int c = 0; c < 32; c += 4)
          *reinterpret_cast<float4*>(S + row * sp + 32 * g + c) =
              make_float4(__uint_as_float(r[c]) * cs2[32 * g + c] * isb,
                          __uint_as_float(r[c + 1]) * cs2[32 * g + c + 1] * isb,
                          __uint_as_float(r[c + 2]) * cs2[32 * g + c + 2] * isb,
                          __uint_as_float(r[c + 3]) * cs2[32 * g + c + 3] * isb);
      }
    }
  }
  if (dir == 1) {
    // the solution update, coalesced: H (round 0), L (round 1), (L, L_lo) +=
    // (later rounds) or the FP64 output (single pass)
    __syncthreads();
    const long long base = (long long)k * nx * ny;
    float* xl = J.xh + P;
    float* xll = J.xh + 2 * P;
    for (int e = tid; e < nx * ny; e += kRT) {
      const int jj = e / nx, ii = e % nx;
      const float w = S[jj * sp + ii];
      const long long p = base + e;
      if (J.single_pass) {
        J.out[p] = (double)w;
      } else if (round == 0) {
        J.xh[p] = w;
      } else if (round == 1) {
        xl[p] = w;
      } else {
        // (L, L_lo) + w: two-sum of the high parts, low parts added, renormalised
        const float oh = xl[p], ol = round >= 3 ? xll[p] : 0.f;
        const float s2 = oh + w;
        const float bb = s2 - oh;
        const float er = (oh - (s2 - bb)) + (w - bb) + ol;
        const float nh = s2 + er;
        xl[p] = nh;
        xll[p] = er - (nh - s2);
      }
    }
  }
  tc::tc_fence_before();
  if (first) {
    // ||b||^2 and the volume-weighted sums of this plane; its solve's last
    // plane resets the status, reduces them and writes the lambda-scaled flux
    // weights
    double w3[3] = {(double)sbb, mean ? df::to_f64(svb) : 0.0, mean ? df::to_f64(sv) : 0.0};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int c = 0; c < 3; ++c) w3[c] += __shfl_down_sync(0xffffffffu, w3[c], o);
    if (lane == 0)
      for (int c = 0; c < 3; ++c) red[3 * warp + c] = w3[c];
    __syncthreads();
    if (tid == 0) {
      double t[3] = {0.0, 0.0, 0.0};
      for (int w = 0; w < kRT / 32; ++w)
        for (int c = 0; c < 3; ++c) t[c] += red[3 * w + c];
      J.partials[4 * k + 0] = 0.0;
      J.partials[4 * k + 1] = t[0];
      J.partials[4 * k + 2] = t[1];
      J.partials[4 * k + 3] = t[2];
    }
  }
  __syncthreads();
  return true;
}

// ---- the first pass's reduction ----

// After the first forward pass: the solve's status reset, ||b||^2, the
// volume-weighted mean of b (zero-flux Laplace problem) and the non-finite
// check from the per-plane partials, and the lambda-scaled flux weights of
// the residual.  One unit per solve in the round-0 Thomas pass.
__device__ void unit_finish0(const ResJob& J, int tid) {
  if (tid == 0) {
    J.st->tol_used = J.tol;
    J.st->refine_steps = 0;
    J.st->iters = 0;
    J.st->error = 0;
  }
  finish_block(J.partials, J.nz, J.st, J.tol, 0, J.singular, tid, kRT);
  const df::F2 lam = df::from_f64(J.lambda);
  for (int d = 0; d < 3; ++d) {
    const int n = d == 0 ? J.nx : (d == 1 ? J.ny : J.nz);
    for (int kind = 0; kind < 3; ++kind)
      for (int e = tid; e < n; e += kRT) {
        const float2 w = J.w[d][kind][e];
        const df::F2 v = df::mul(lam, df::make(w.x, w.y));
        J.lam_w[(d * 3 + kind) * kMaxN + e] = make_float2(v.hi, v.lo);
      }
  }
  __syncthreads();
}

// ---- T: Thomas sweep along z ----

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// One thread per (x-mode i, y-mode j) line of the spectral planes: solve
// (s M_z - lambda K_z) u = M_z f with s = sigma - lambda (Lambda_x,i +
// Lambda_y,j) (Sec. 3, end).  A unit copies its J.lt consecutive lines (all
// planes) into shared memory at once, sweeps there (d' in place, c' beside
// it) and writes the lines back.  The line of the zero-flux Laplacian with
// Lambda = 0 is singular: its right side is projected to zero M_z-weighted
// mean, u_0 pinned to 0, rows 1.. solved and the weighted mean of the solution
// removed.
__device__ void unit_thomas(const ResJob& J, int tile, float* sm, int tid) {
  const int nz = J.nz, lt = J.lt, g = lt / 4;
  const float lam = (float)J.lambda;
  float* tf = sm;                                              // [nz][lt]: f, then d', then u
  float* tc = sm + nz * lt;                                    // [nz][lt]: c'
  float4* co = reinterpret_cast<float4*>(sm + 2 * nz * lt);    // [nz]: {M_k, lambda Kd_k, lower, upper}
  const long long pl = (long long)J.ny * J.px;
  const int lines = J.ny * J.px, l0 = tile * lt;
  for (int e = tid; e < nz * g; e += kRT) {
    const int k = e / g, c = (e % g) * 4;
    if (l0 + c < lines)
      cp16(tf + k * lt + c, J.F + k * pl + l0 + c);
    else
      *reinterpret_cast<float4*>(tf + k * lt + c) = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int k = tid; k < nz; k += kRT)
    co[k] = make_float4(J.mz[k], lam * J.kdz[k], k > 0 ? -lam * J.koz[k - 1] : 0.f,
                        k + 1 < nz ? -lam * J.koz[k] : 0.f);
  const int l = l0 + tid;
  const int i = l % J.px, j = l / J.px;
  const bool mine = tid < lt && j < J.ny && i < J.nx;
  double lab = 0.0;
  if (mine) lab = J.lamx[i] + J.lamy[j];
  cp_wait_all();
  __syncthreads();
  if (mine) {
    float* f = tf + tid;
    float* c = tc + tid;
    const float s = (float)(J.sigma - J.lambda * lab);
    if (!(J.singular && lab == 0.0)) {
      // blocks of 8 planes: the next block's values are read before the
      // current block's results are stored, so no shared-memory load sits on
      // the recurrence
      float cp = 0.f, dp = 0.f;
      float fv[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) fv[e] = e < nz ? f[e * lt] : 0.f;
      for (int k0 = 0; k0 < nz; k0 += 8) {
        float fn[8], dv[8], cv[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) fn[e] = k0 + 8 + e < nz ? f[(k0 + 8 + e) * lt] : 0.f;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float4 q = co[min(k0 + e, nz - 1)];
          const float inv = rcp_approx(fmaf(-q.z, cp, fmaf(s, q.x, -q.y)));
          const float cn = q.w * inv;
          const float dn = fmaf(q.x, fv[e], -q.z * dp) * inv;
          if (k0 + e < nz) {
            cp = cn;
            dp = dn;
          }
          dv[e] = dp;
          cv[e] = cp;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (k0 + e < nz) {
            f[(k0 + e) * lt] = dv[e];
            c[(k0 + e) * lt] = cv[e];
          }
#pragma unroll
        for (int e = 0; e < 8; ++e) fv[e] = fn[e];
      }
      // back substitution (c'_{nz-1} = 0: u_{nz-1} = d'_{nz-1}), blocks of 8
      // planes downwards, read ahead the same way
      float u = dp;
      float dv[8], cv[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = nz - 2 - e;
        dv[e] = k >= 0 ? f[k * lt] : 0.f;
        cv[e] = k >= 0 ? c[k * lt] : 0.f;
      }
      for (int k1 = nz - 2; k1 >= 0; k1 -= 8) {
        float dn[8], cn[8], uv[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int k = k1 - 8 - e;
          dn[e] = k >= 0 ? f[k * lt] : 0.f;
          cn[e] = k >= 0 ? c[k * lt] : 0.f;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          u = k1 - e >= 0 ? fmaf(-cv[e], u, dv[e]) : u;
          uv[e] = u;
        }
#pragma unroll
        for (int e = 0; e < 8; ++e)
          if (k1 - e >= 0) f[(k1 - e) * lt] = uv[e];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          dv[e] = dn[e];
          cv[e] = cn[e];
        }
      }
    } else {
      float smz = 0.f, sf = 0.f;
      for (int k = 0; k < nz; ++k) {
        smz += co[k].x;
        sf = fmaf(co[k].x, f[k * lt], sf);
      }
      const float mu = sf / smz;
      float cp = 0.f, dp = 0.f;
      for (int k = 1; k < nz; ++k) {
        const float4 q = co[k];
        const float lo = k > 1 ? q.z : 0.f;
        const float inv = rcp_approx(fmaf(-lo, cp, fmaf(s, q.x, -q.y)));
        cp = q.w * inv;
        dp = fmaf(q.x, f[k * lt] - mu, -lo * dp) * inv;
        f[k * lt] = dp;
        c[k * lt] = cp;
      }
      float u = dp, su = co[nz - 1].x * dp;
      for (int k = nz - 2; k >= 1; --k) {
        u = fmaf(-c[k * lt], u, f[k * lt]);
        f[k * lt] = u;
        su = fmaf(co[k].x, u, su);
      }
      f[0] = 0.f;
      const float mean = su / smz;
      for (int k = 0; k < nz; ++k) f[k * lt] = f[k * lt] - mean;
    }
  }
  __syncthreads();
  for (int e = tid; e < nz * g; e += kRT) {
    const int k = e / g, c = (e % g) * 4;
    if (l0 + c < lines)
      *reinterpret_cast<float4*>(J.F + k * pl + l0 + c) = *reinterpret_cast<const float4*>(tf + k * lt + c);
  }
  __syncthreads();
}

// ---- R: residual ----

template <int MODE, bool LO, bool MEAN, bool OUT, bool FAST>
__device__ __noinline__ void resid_v(const ResidArgs& a, double* sh, int bx, int by, int bz, int bid, bool vec) {
  if (vec)
    resid_body<MODE, 2, LO, MEAN, OUT, false, true, FAST>(a, sh, bx, by, bz, bid);
  else
    resid_body<MODE, 2, LO, MEAN, OUT, false, false, FAST>(a, sh, bx, by, bz, bid);
}

// L1 prefetch of the lines a box of rows touches (k, j, i inclusive ranges;
// rows of `pitch` elements, planes of `plane`): every line of a residual
// unit's footprint is requested at once, so its z-march finds them on chip
__device__ __forceinline__ void pf_line(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

template <typename T>
__device__ __forceinline__ void pf_box(const T* base, int pitch, long long plane, int k0, int k1, int j0, int j1, int i0,
                                       int i1, int tid) {
  const int nj = j1 - j0 + 1, rows = (k1 - k0 + 1) * nj;
  const int lpr = (int)(((i1 - i0 + 1) * sizeof(T) + 127) / 128) + 1;
  for (int t = tid; t < rows * lpr; t += kRT) {
    const int r = t / lpr, li = t % lpr;
    const T* row = base + (long long)(k0 + r / nj) * plane + (long long)(j0 + r % nj) * pitch;
    const char* a = reinterpret_cast<const char*>((reinterpret_cast<uintptr_t>(row + i0) & ~(uintptr_t)127) + 128 * li);
    if (a <= reinterpret_cast<const char*>(row + i1)) pf_line(a);
  }
}

__device__ void unit_resid(const ResJob& J, int round, int rb, int tid, double* sh, unsigned* s_last) {
  const long long P = (long long)J.nx * J.ny * J.nz;
  ResidArgs a;
  a.nx = J.nx;
  a.ny = J.ny;
  a.nz = J.nz;
  for (int d = 0; d < 3; ++d) {
    a.wp[d] = J.lam_w + (d * 3 + 0) * kMaxN;
    a.wm[d] = J.lam_w + (d * 3 + 1) * kMaxN;
    a.w0[d] = J.lam_w + (d * 3 + 2) * kMaxN;
    a.m[d] = J.m[d];
  }
  a.wy = nullptr;
  a.fast_limit = J.fast_limit;
  const df::F2 sg = df::from_f64(J.sigma), lm = df::from_f64(J.lambda);
  a.sigma = make_float2(sg.hi, sg.lo);
  a.lambda = make_float2(lm.hi, lm.lo);
  a.sig_mode = 2;
  a.b = J.b;
  a.xh = J.xh;
  a.xl = J.xh + P;
  a.xll = J.xh + 2 * P;
  a.r1 = J.r1;
  a.r1_lo = J.r1 + J.r1_plane;
  a.r = round == 0 ? J.r1 : J.r;
  a.r_lo = J.r1 + J.r1_plane;
  a.r_pitch = J.px;
  a.zchunk = J.zchunk;
  a.out = J.out;
  a.rmax = J.rmax;
  a.st = J.st;
  a.sub_mean = 0;
  a.want_mean = 0;
  a.partials = J.partials;
  a.fin = FinishArgs{nullptr, nullptr, nullptr, 0.0, 0, 0, 0};
  const int bx = rb % J.rgx, by = (rb / J.rgx) % J.rgy, bz = rb / (J.rgx * J.rgy);
  const bool vec = J.vec != 0;
  {
    // the unit's footprint: the solution planes with a one-cell halo, the
    // right-hand side part (b or r_1) and H without
    const int nx = J.nx, ny = J.ny, nz = J.nz;
    const int i0 = bx * kResBX, i1 = min(i0 + kResBX - 1, nx - 1);
    const int j0 = by * kResTY, j1 = min(j0 + kResTY - 1, ny - 1);
    const int k0 = bz * J.zchunk, k1 = min(k0 + J.zchunk - 1, nz - 1);
    const int hi0 = max(i0 - 1, 0), hi1 = min(i1 + 1, nx - 1), hj0 = max(j0 - 1, 0), hj1 = min(j1 + 1, ny - 1);
    const int hk0 = max(k0 - 1, 0), hk1 = min(k1 + 1, nz - 1);
    const long long pn = (long long)nx * ny, pr = (long long)ny * J.px;
    if (round == 0) {
      pf_box(J.xh, nx, pn, hk0, hk1, hj0, hj1, hi0, hi1, tid);
      pf_box(J.b, nx, pn, k0, k1, j0, j1, i0, i1, tid);
    } else {
      pf_box(J.xh + P, nx, pn, hk0, hk1, hj0, hj1, hi0, hi1, tid);
      if (round >= 2) pf_box(J.xh + 2 * P, nx, pn, hk0, hk1, hj0, hj1, hi0, hi1, tid);
      pf_box(J.xh, nx, pn, k0, k1, j0, j1, i0, i1, tid);
      pf_box(J.r1, J.px, pr, k0, k1, j0, j1, i0, i1, tid);
      pf_box(J.r1 + J.r1_plane, J.px, pr, k0, k1, j0, j1, i0, i1, tid);
    }
  }
  if (round == 0) {
    if (J.singular)
      resid_v<0, false, true, false, false>(a, sh, bx, by, bz, rb, vec);
    else
      resid_v<0, false, false, false, false>(a, sh, bx, by, bz, rb, vec);
  } else if (J.singular) {
    if (round >= 2)
      resid_v<1, true, true, false, false>(a, sh, bx, by, bz, rb, vec);
    else
      resid_v<1, false, true, false, false>(a, sh, bx, by, bz, rb, vec);
  } else {
    // plain FP32 correction residual when the first residual bounds its error
    const bool fast = J.fast_limit > 0.0 && J.st->scal[1] <= J.fast_limit;
    if (round >= 2) {
      if (fast)
        resid_v<1, true, false, true, true>(a, sh, bx, by, bz, rb, vec);
      else
        resid_v<1, true, false, true, false>(a, sh, bx, by, bz, rb, vec);
    } else {
      if (fast)
        resid_v<1, false, false, true, true>(a, sh, bx, by, bz, rb, vec);
      else
        resid_v<1, false, false, true, false>(a, sh, bx, by, bz, rb, vec);
    }
  }
  if (last_unit(J, J.rgx * J.rgy * J.rgz, tid, s_last)) {
    finish_block(J.partials, J.rgx * J.rgy * J.rgz, J.st, J.tol, round == 0 ? 1 : 2, J.singular, tid, kRT);
    if (tid == 0) *J.ticket = 0u;
  }
  __syncthreads();
}

// ---- output of solves that end without a refinement step, or singular ----

__device__ void unit_out(const ResJob& J, int chunk, int tid) {
  const long long P = (long long)J.nx * J.ny * J.nz;
  const int steps = J.st->refine_steps;
  const bool has_l = steps > 0, has_ll = steps > 1;
  df::F2 mu = df::make(0.f, 0.f);
  if (J.singular) mu = df::from_f64(J.st->scal[0]);
  const float* xl = J.xh + P;
  const float* xll = J.xh + 2 * P;
  const long long p0 = (long long)chunk * kOutChunk;
  for (int e = tid; e < kOutChunk; e += kRT) {
    const long long p = p0 + e;
    if (p >= P) break;
    df::F2 u = df::two_sum(J.xh[p], has_l ? xl[p] : 0.f);
    if (has_ll) u = df::fast_two_sum(u.hi, u.lo + xll[p]);
    if (J.singular) u = df::sub(u, mu);
    J.out[p] = df::to_f64_bits(u);
  }
}

// ---- the kernel ----

__global__ void __launch_bounds__(kRT, 2) k_resident(const __grid_constant__ ResLaunch L) {
  extern __shared__ __align__(1024) uint8_t res_smem[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(res_smem) + 1023) & ~(uintptr_t)1023);
  float* sm = reinterpret_cast<float*>(base);
  const PlaneSmem ps{base, base + res_s_bytes(L.cls), base + res_s_bytes(L.cls) + res_a_bytes(L.cls)};
  __shared__ double sh[4 * kResTY];
  __shared__ double red[3 * (kRT / 32)];
  __shared__ float redf[kRT / 32];
  __shared__ int s_ok;
  __shared__ volatile int s_abort;
  __shared__ unsigned s_last;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_mbar;
  __shared__ unsigned char active[kResMaxJobs];
  __shared__ __align__(16) ResJob s_job;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  // tensor memory for the plane products (128 columns) and their completion barrier
  if (tid < 32) {
    tc::tmem_alloc(&s_tmem, 128);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&s_mbar, 1);
    tc::fence_mbar_init();
    s_abort = 0;
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tbase = s_tmem;
  uint32_t mph = 0;
  // every unit of one pass, round-robin over the CTAs; a unit reads its
  // solve's descriptor from a shared-memory copy (the parameter block is
  // indexed by the solve, and its reads would each wait on the constant cache)
  int s_jq = -1;
  auto pass = [&](int kind, auto&& fn) {
    const int total = units_total(L, active, kind);
    for (int u = blockIdx.x; u < total; u += gridDim.x) {
      int q = 0, loc = 0;
      unit_of(L, active, kind, u, &q, &loc);
      if (q != s_jq) {
        __syncthreads();
        const int* src = reinterpret_cast<const int*>(&L.job[q]);
        int* dst = reinterpret_cast<int*>(&s_job);
        for (int e = tid; e < (int)(sizeof(ResJob) / sizeof(int)); e += kRT) dst[e] = src[e];
        __syncthreads();
        s_jq = q;
      }
      fn(s_job, loc);
    }
  };
  // a plane pass; a tensor-memory wait that ran out aborts the launch
  auto plane_pass = [&](int dir, int round) {
    pass(U_PLANE, [&](const ResJob& J, int k) {
      if (s_abort) return;
      if (!unit_plane(J, dir, round, k, ps, tbase, &s_mbar, mph, tid, redf, red, &s_last, &s_abort, L.wait) &&
          tid == 0) {
        atomicExch(L.bar + 2, 1u);
        atomicExch(L.err, 9);
      }
    });
  };
  auto set_active = [&](auto&& pred) {
    __syncthreads();
    if (tid < L.njobs) active[tid] = pred(L.job[tid]) ? 1 : 0;
    __syncthreads();
  };
  set_active([](const ResJob&) { return true; });
  // round 0: the first direct solve of every solve of the launch
  plane_pass(0, 0);
  bool ok = grid_barrier(L, tid, &s_ok);
  if (ok) {
    pass(U_LINES0, [&](const ResJob& J, int t) {
      if (t < (J.ny * J.px + J.lt - 1) / J.lt)
        unit_thomas(J, t, sm, tid);
      else
        unit_finish0(J, tid);
    });
    ok = grid_barrier(L, tid, &s_ok);
  }
  if (ok) plane_pass(1, 0);
  if (ok && L.max_rounds >= 0) {
    // residual check of the refined solves, then the refinement rounds
    ok = grid_barrier(L, tid, &s_ok);
    set_active([](const ResJob& J) { return J.single_pass == 0; });
    if (ok) {
      pass(U_RESID, [&](const ResJob& J, int rb) { unit_resid(J, 0, rb, tid, sh, &s_last); });
      ok = grid_barrier(L, tid, &s_ok);
    }
    for (int round = 1; ok && round <= L.max_rounds; ++round) {
      set_active([&](const ResJob& J) {
        return J.single_pass == 0 && round <= J.max_refine &&
               *reinterpret_cast<volatile const int*>(&J.st->done) == 0;
      });
      if (units_total(L, active, U_PLANE) == 0) break;
      plane_pass(0, round);
      if (!(ok = grid_barrier(L, tid, &s_ok))) break;
      pass(U_LINES, [&](const ResJob& J, int t) { unit_thomas(J, t, sm, tid); });
      if (!(ok = grid_barrier(L, tid, &s_ok))) break;
      plane_pass(1, round);
      if (!(ok = grid_barrier(L, tid, &s_ok))) break;
      pass(U_RESID, [&](const ResJob& J, int rb) { unit_resid(J, round, rb, tid, sh, &s_last); });
      ok = grid_barrier(L, tid, &s_ok);
    }
    if (ok) {
      // FP64 output where no correction pass wrote it: convergence in round 0
      // (L = 0), and the zero-flux Laplace problem (minus the volume-weighted
      // mean of the solution)
      set_active([](const ResJob& J) {
        return J.single_pass == 0 &&
               (J.singular || *reinterpret_cast<volatile const int*>(&J.st->refine_steps) == 0);
      });
      pass(U_OUT, [&](const ResJob& J, int c) { unit_out(J, c, tid); });
    }
  }
  // an MMA batch whose wait ran out completes before its tensor memory is freed
  if (s_abort && tid == 0) tc::mbar_drain(&s_mbar, mph);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (tid < 32) tc::tmem_dealloc(tbase, 128);
  grid_exit(L, tid);
}

size_t resident_smem(int cls) { return (size_t)(1024 + res_s_bytes(cls) + res_a_bytes(cls) + res_b_bytes(cls)); }

}  // namespace

fdi_status resident_launch(fdi_plan* owner, const ResJob* jobs, int n, cudaStream_t s) {
  if (n <= 0) return FDI_OK;
  if (n > kResMaxJobs) {
    set_error("too many solves for one resident launch");
    return FDI_ERR_INVALID_ARG;
  }
  static ResLaunch L;  // host staging (the launch copies the parameter block)
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  L.njobs = n;
  L.max_rounds = -1;
  int cls = 64;
  long long units = 1;
  long long u_plane = 0, u_lines = 0, u_resid = 0;
  for (int q = 0; q < n; ++q) {
    L.job[q] = jobs[q];
    cls = std::max(cls, jobs[q].cls);
    if (!jobs[q].single_pass) L.max_rounds = std::max(L.max_rounds, jobs[q].max_refine);
    u_plane += jobs[q].nz;
    u_resid += (long long)jobs[q].rgx * jobs[q].rgy * jobs[q].rgz;
  }
  // Thomas lines per unit: the largest power of two <= 256 whose tile (f and
  // c', all planes, and the z coefficients) fits the launch's shared memory
  const size_t smem_b = resident_smem(cls) - 1024;
  u_lines = 0;
  for (int q = 0; q < n; ++q) {
    const int nz = jobs[q].nz;
    int lt = 256;
    while (lt > 4 && (size_t)8 * nz * lt + 16 * (size_t)nz > smem_b) lt /= 2;
    L.job[q].lt = lt;
    u_lines += (jobs[q].ny * jobs[q].px + lt - 1) / lt + 1;
  }
  units = std::max(u_plane, std::max(u_lines, u_resid));
  L.cls = cls;
  L.bar = owner->res_bar;
  L.err = owner->d_err;
  L.wait = owner->wait_cycles > 0 ? owner->wait_cycles : tc::kWaitCycles;
  const size_t smem = resident_smem(cls);
  int dev = 0, sms = 0, occ = 0;
  FDI_CUDA_TRY(cudaGetDevice(&dev));
  FDI_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // the attribute follows the launch's own size: a larger one would keep the
  // occupancy calculation (and the cooperative grid) at one CTA per SM
  static size_t smem_set = 0;
  if (smem_set == 0)
    FDI_CUDA_TRY(cudaFuncSetAttribute(k_resident, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared));
  if (smem != smem_set) {
    FDI_CUDA_TRY(cudaFuncSetAttribute(k_resident, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    smem_set = smem;
  }
  FDI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_resident, kRT, smem));
  if (occ < 1) {
    set_error("resident solve: no CTA fits on an SM");
    return FDI_ERR_CUDA;
  }
  const unsigned grid = (unsigned)std::min<long long>((long long)occ * sms, units);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(32, kRT / 32);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  FDI_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_resident, L));
  FDI_LAUNCH_CHECK(owner);
  return FDI_OK;
}

}  // namespace fdi
