// Double-float residual of the mixed-precision solve (flux form of Eq. 23)
// and the fixed-order reduction behind its convergence check; shared by the
// pass-by-pass solve (mixed.cu) and the resident small-grid solve
// (resident.cu).
#pragma once
#include <cuda_runtime.h>

#include "df.cuh"
#include "fdi_internal.h"

namespace fdi {
namespace {

// fused final reduction (see finish_if_last)
struct FinishArgs {
  unsigned* counter;    // zero between launches
  const double* partials;
  DevStatus* st;
  double tol;
  int kind, want_mean;
  // captured solves: condition of the next refinement round's graph node
  // (set to "not converged"); 0 when running eagerly
  cudaGraphConditionalHandle next_round = 0;
};

struct ResidArgs {
  int nx, ny, nz;
  const float2* wp[3];
  const float2* wm[3];
  const float2* w0[3];
  const float2* m[3];
  const float2* wy;     // periodic-y plans: lambda-scaled y flux weight per plane (null otherwise)
  double fast_limit;    // MODE 1: plain FP32 body when ||r_1|| / ||b|| <= fast_limit (0: never)
  float2 sigma, lambda;
  int sig_mode;         // 0: sigma = 0, 1: sigma = 1, 2: general sigma
  const double* b;
  const float* xh;      // solution planes: H, L (= Lh) and the low plane of L
  const float* xl;
  const float* xll;
  const float* r1;      // r_1 as a double-float pair of planes (MODE 1 input)
  const float* r1_lo;
  float* r;             // FP32 residual (the next solve's input)
  float* r_lo;          // MODE 0: low plane of r_1
  int r_pitch;
  int zchunk;           // planes per block (resid_grid)
  double* out;          // FP64 solution output (null: not written)
  float* rmax;          // atomic max |r|
  const DevStatus* st;
  int sub_mean;
  int want_mean;        // accumulate sum V b and sum V (first pass) or sum V x (later passes)
  double* partials;     // per block: sum r^2, sum b^2, sum V b (or V x), sum V
  FinishArgs fin;
};


__device__ __forceinline__ df::F2 ld2(const float2* p) {
  float2 v = *p;
  return df::make(v.x, v.y);
}

// z-marching residual: a block of 32 (x) x 8 (y) threads covers 64 x 8
// columns; each thread a pair of x-neighbours (i0, i0 + 1) of one row j, over a
// range of planes.  Per plane a thread holds its pair at planes k and k + 1 and
// the pairs of rows j - 1 and j + 1 at plane k (the loads of the next plane
// are issued before the current one is computed; with VEC one 8-byte access
// per pair); the x face inside the pair is differenced once for both points,
// the z face below is the previous plane's upper face, and the x neighbours
// outside the pair come from the neighbouring lanes.  Walls need no branch:
// the flux weights are zero across a wall and the clamped neighbour index
// gives an exact zero difference there; only the Dirichlet wall term (nonzero
// next to a wall) is added under a per-thread flag.  Work per block is fixed,
// so the reduction order is too.
//
// Arithmetic: x = xh + xl (double-float).  With the flux weights already
// multiplied by lambda (w' = lambda w, double-float), lambda L x = L'xh + L'xl;
// each flux of L'xh is formed exactly (two-difference of the float values,
// FMA two-product with the weight's high part) and its high part summed with
// two-sum; the rounding errors, the products with the weights' low parts and
// with the differences' low parts go straight into the FP32 companion sum by
// FMA; L'xl is plain FP32 (it is 2^-24 smaller).  b and -sigma x enter the
// same accumulator, and the FP32 residual is its rounded value: r is stored in
// FP32, so only the cancellation inside the sum needs the extra precision.
//
// CYL: the y direction is periodic (rows wrap around) and its flux weight is
// one value per plane, wy[k] (the cylindrical theta direction, whose flux
// carries the radial factor of the plane).
constexpr int kResTX = 32, kResTY = 8, kResZChunk = 16;  // planes per block (at most)
constexpr int kResBX = 2 * kResTX;                       // x columns per block

struct Acc {
  float h, l;  // unnormalised double-float accumulator
};

__device__ __forceinline__ void acc_add(Acc& s, float ph, float pl) {
  const float t = s.h + ph;
  const float bb = t - s.h;
  s.l += ((s.h - (t - bb)) + (ph - bb)) + pl;
  s.h = t;
}

// a - c = d + dl exactly (Knuth two-difference)
struct Diff {
  float d, dl;
};

__device__ __forceinline__ Diff two_diff(float a, float c) {
  const float d = a - c;
  const float bb = d - a;
  return Diff{d, (a - (d - bb)) - (c + bb)};
}

__device__ __forceinline__ Diff neg(Diff t) { return Diff{-t.d, -t.dl}; }

// s += w * (d + dl) for a double-float weight w: the high product enters by
// two-sum, its exact rounding error and the two small cross products by FMA
// into the low part
__device__ __forceinline__ void acc_flux(Acc& s, float2 w, Diff t) {
  const float p = w.x * t.d;
  const float e = fmaf(w.x, t.d, -p);
  const float tt = s.h + p;
  const float bb = tt - s.h;
  float l = fmaf(w.x, t.dl, s.l);
  l = fmaf(w.y, t.d, l);
  s.l = l + (((s.h - (tt - bb)) + (p - bb)) + e);
  s.h = tt;
}

// Plain FP32 forms of the same steps, for the correction residual when the
// first residual is small (FAST): the difference rounded once, the flux
// product added by FMA to the high part, other terms added in FP32.
template <bool FAST>
__device__ __forceinline__ Diff diff_of(float a, float c) {
  if (FAST) return Diff{a - c, 0.f};
  return two_diff(a, c);
}

template <bool FAST>
__device__ __forceinline__ void flux_of(Acc& s, float2 w, Diff t) {
  if (FAST)
    s.h = fmaf(w.x, t.d, s.h);
  else
    acc_flux(s, w, t);
}

template <bool FAST>
__device__ __forceinline__ void add_of(Acc& s, float ph, float pl) {
  if (FAST) {
    s.h += ph;
    s.l += pl;
  } else {
    acc_add(s, ph, pl);
  }
}

// one x pair of FP32 values (hi) and, for LO, of the low plane
struct Pair {
  float a, b;     // points i0, i0 + 1
  float la, lb;   // low parts (LO only)
};

template <bool VEC, bool LO>
__device__ __forceinline__ Pair ld_pair(const float* hi, const float* lo, int o, int d1) {
  Pair v{0.f, 0.f, 0.f, 0.f};
  if (VEC) {
    const float2 h = *reinterpret_cast<const float2*>(hi + o);
    v.a = h.x;
    v.b = h.y;
    if (LO) {
      const float2 l = *reinterpret_cast<const float2*>(lo + o);
      v.la = l.x;
      v.lb = l.y;
    }
  } else {
    v.a = hi[o];
    v.b = hi[o + d1];
    if (LO) {
      v.la = lo[o];
      v.lb = lo[o + d1];
    }
  }
  return v;
}

// Two residual passes share this body.
//   MODE 0 (after the first solve):  r_1 = b - A H, with H exactly FP32; the
//     result is stored as a double-float pair (r_hi, r_lo) of FP32 planes and
//     r_hi is the next solve's input.
//   MODE 1 (after every correction): r = r_1 - A L, with L = Lh (+ Ll when LO)
//     the accumulated corrections; A is linear, so this equals b - A (H + L)
//     exactly, and only the small field L passes through the stencil.
// SIG: 0 sigma = 0, 1 sigma = 1, 2 general sigma.  MEAN: zero-flux Laplace
// problem (MODE 0 subtracts the volume-weighted mean of b; volume-weighted
// sums of the solution H (+ L) are reduced).  OUT: write the FP64 solution
// H + L.  VEC: nx even and 16-byte aligned FP64 arrays, pairs moved by vector
// accesses.
template <int MODE, int SIG, bool LO, bool MEAN, bool OUT, bool CYL, bool VEC, bool FAST>
__device__ __forceinline__ void resid_body(const ResidArgs& a, double* sh, int bx, int by, int bz, long long bid) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int lane = threadIdx.x, wy = threadIdx.y;
  const int i0 = 2 * (bx * kResTX + lane);
  const int j = by * kResTY + wy;
  const int k0 = bz * a.zchunk, k1 = min(nz, k0 + a.zchunk);
  const bool act0 = j < ny && i0 < nx, act1 = j < ny && i0 + 1 < nx;
  // clamped indices keep every load in bounds; a clamped neighbour is the
  // point itself (zero difference) and its flux weight is zero (a wall)
  const int ia = VEC ? min(i0, nx - 2) : min(i0, nx - 1);
  const int d1 = (VEC || ia + 1 < nx) ? 1 : 0;  // second point of the pair (scalar path)
  const int jc = min(j, ny - 1);
  const int js = jc > 0 ? jc - 1 : (CYL ? ny - 1 : 0);
  const int jn = jc + 1 < ny ? jc + 1 : (CYL ? 0 : ny - 1);
  // x of the value lane 31 needs east of its pair and lane 0 west of its pair
  const int ie = lane == kResTX - 1 ? min(i0 + 2, nx - 1) : (lane == 0 ? max(i0 - 1, 0) : ia);
  const long long oc = (long long)jc * nx + ia, os = (long long)js * nx + ia, on = (long long)jn * nx + ia;
  const long long oe = (long long)jc * nx + ie;
  const long long orr_ = (long long)jc * a.r_pitch + ia;
  float mean_h = 0.f, mean_l = 0.f;
  if (MODE == 0 && MEAN) {
    const df::F2 mb = df::from_f64(a.st->mean_b);
    mean_h = -mb.hi;
    mean_l = -mb.lo;
  }
  const int ib = ia + d1;
  const float2 wpxa = a.wp[0][ia], wmxa = a.wm[0][ia], wpxb = a.wp[0][ib], wmxb = a.wm[0][ib];
  float2 wpy = make_float2(0.f, 0.f), wmy = wpy;
  float2 w0y = make_float2(0.f, 0.f);
  if (!CYL) {
    wpy = a.wp[1][jc];
    wmy = a.wm[1][jc];
    w0y = a.w0[1][jc];
  }
  const float2 w0xa = a.w0[0][ia], w0xb = a.w0[0][ib];
  const bool wall_xy = w0xa.x != 0.f || w0xb.x != 0.f || w0y.x != 0.f;
  df::F2 Va = df::make(0.f, 0.f), Vb = Va;
  if (MEAN) {
    const df::F2 my = ld2(a.m[1] + jc);
    Va = df::mul(ld2(a.m[0] + ia), my);
    Vb = df::mul(ld2(a.m[0] + ib), my);
  }
  float srr = 0.f, sbb = 0.f, rmax = 0.f;
  df::F2 svb = df::make(0.f, 0.f), sv = df::make(0.f, 0.f);
  // Per-row base pointers and 32-bit plane offsets (every field has fewer
  // than 2^31 elements): each access is one wide multiply-add.
  const int szi = nx * ny;           // plane stride of the [z][y][x] fields
  const int rsi = ny * a.r_pitch;    // plane stride of the residual planes
  // the field the stencil acts on: H (MODE 0) or L (MODE 1), (hi, lo) planes
  const float* uh = MODE == 0 ? a.xh : a.xl;
  const float* ul = (MODE == 1 && LO) ? a.xll : uh;
  const float* uhc = uh + oc;
  const float* uhs = uh + os;
  const float* uhn = uh + on;
  const float* uhe = uh + oe;
  const float* ulc = ul + oc;
  const float* uls = ul + os;
  const float* uln = ul + on;
  const float* ule = ul + oe;
  const double* bc = MODE == 0 ? a.b + oc : nullptr;
  const float* q1h = MODE == 1 ? a.r1 + orr_ : nullptr;
  const float* q1l = MODE == 1 ? a.r1_lo + orr_ : nullptr;
  const float* hc = (MODE == 1 && (OUT || MEAN)) ? a.xh + oc : nullptr;
  float* rc = a.r + orr_;
  float* rlc = MODE == 0 ? a.r_lo + orr_ : nullptr;
  double* outc = OUT ? a.out + oc : nullptr;
  constexpr bool LOM = MODE == 1 && LO;
  auto ldp = [&](const float* h, const float* l, int o) { return ld_pair<VEC, LOM>(h, l, o, d1); };
  auto lde = [&](int o, float& l) {
    if (LOM) l = ule[o];
    return uhe[o];
  };
  // plane k's right-hand side part: b (MODE 0, FP64) or r_1 (MODE 1, hi and lo)
  auto ldb = [&](int o, double& b0, double& b1) {
    if (VEC) {
      const double2 v = *reinterpret_cast<const double2*>(bc + o);
      b0 = v.x;
      b1 = v.y;
    } else {
      b0 = bc[o];
      b1 = bc[o + d1];
    }
  };
  auto ldr1 = [&](int o, Pair& q) { q = ld_pair<VEC, true>(q1h, q1l, o, d1); };
  auto ldh = [&](int o, float& h0, float& h1) {
    const Pair q = ld_pair<VEC, false>(hc, nullptr, o, d1);
    h0 = q.a;
    h1 = q.b;
  };
  // pipeline: pair C at plane k and P at k + 1, rows below (S) and above (N)
  // and the edge value E at plane k, and the right-hand side parts of plane k
  int ok = k0 * szi;                                 // plane k of the fields
  int rk = k0 * rsi;                                 // plane k of the residual planes
  Pair C = ldp(uhc, ulc, ok);
  Pair P = ldp(uhc, ulc, min(k0 + 1, nz - 1) * szi);
  Pair S = ldp(uhs, uls, ok), N = ldp(uhn, uln, ok);
  float El = 0.f;
  float E = lde(ok, El);
  double b0 = 0.0, b1 = 0.0;
  Pair Q{0.f, 0.f, 0.f, 0.f};
  float h0 = 0.f, h1 = 0.f;
  if (MODE == 0) ldb(ok, b0, b1);
  if (MODE == 1) ldr1(rk, Q);
  if (MODE == 1 && (OUT || MEAN)) ldh(ok, h0, h1);
  // exact z differences of the faces below plane k (u_{k-1} - u_k) and the
  // low parts of plane k-1 (LO); at k = 0 the clamped plane gives zero
  Diff dza, dzb;
  float mla = 0.f, mlb = 0.f;
  {
    const Pair M = ldp(uhc, ulc, max(k0 - 1, 0) * szi);
    dza = diff_of<FAST>(M.a, C.a);
    dzb = diff_of<FAST>(M.b, C.b);
    mla = M.la;
    mlb = M.lb;
  }
  const float2* wpz = a.wp[2];
  const float2* wmz = a.wm[2];
  const float2* w0z = a.w0[2];
  // two planes per loop pass let the register pipeline rotate without moves;
  // the exact and low-plane correction bodies keep one (their registers would
  // spill at the correction kernel's occupancy)
  constexpr int kUnroll = (MODE == 1 && (LO || !FAST)) ? 1 : 2;
#pragma unroll kUnroll
  for (int k = k0; k < k1; ++k) {
    // loads of the next plane (block-uniform guard)
    Pair P2 = P, S2 = S, N2 = N, Q2 = Q;
    float E2 = E, E2l = El;
    double b02 = 0.0, b12 = 0.0;
    float h02 = 0.f, h12 = 0.f;
    if (k + 1 < k1) {
      const int o1 = ok + szi;
      P2 = ldp(uhc, ulc, k + 2 < nz ? o1 + szi : o1);
      S2 = ldp(uhs, uls, o1);
      N2 = ldp(uhn, uln, o1);
      E2 = lde(o1, E2l);
      if (MODE == 0) ldb(o1, b02, b12);
      if (MODE == 1) ldr1(rk + rsi, Q2);
      if (MODE == 1 && (OUT || MEAN)) ldh(o1, h02, h12);
    }
    // x neighbours outside the pair: from the neighbouring lanes, or the edge value
    const float sd = __shfl_down_sync(0xffffffffu, C.a, 1);
    const float su = __shfl_up_sync(0xffffffffu, C.b, 1);
    const float eb = lane == kResTX - 1 ? E : sd;   // east of point b
    const float wa = lane == 0 ? E : su;            // west of point a
    float ebl = 0.f, wal = 0.f;
    if (MODE == 1 && LO) {
      const float sdl = __shfl_down_sync(0xffffffffu, C.la, 1);
      const float sul = __shfl_up_sync(0xffffffffu, C.lb, 1);
      ebl = lane == kResTX - 1 ? El : sdl;
      wal = lane == 0 ? El : sul;
    }
    Acc Sa, Sb;
    df::F2 ba = df::make(0.f, 0.f), bb = ba;
    if (MODE == 0) {
      ba = df::from_f64(b0);
      bb = df::from_f64(b1);
      Sa = Acc{ba.hi, ba.lo};
      Sb = Acc{bb.hi, bb.lo};
      if (MEAN) {
        add_of<FAST>(Sa, mean_h, mean_l);
        add_of<FAST>(Sb, mean_h, mean_l);
      }
    } else {
      Sa = Acc{Q.a, Q.la};
      Sb = Acc{Q.b, Q.lb};
    }
    if (MEAN) {
      const df::F2 mz = ld2(a.m[2] + k);
      const df::F2 Vka = df::mul(Va, mz), Vkb = df::mul(Vb, mz);
      df::F2 xa = df::make(C.a, 0.f), xb = df::make(C.b, 0.f);
      if (MODE == 1) {
        xa = df::two_sum(h0, C.a);
        xa = df::fast_two_sum(xa.hi, xa.lo + C.la);
        xb = df::two_sum(h1, C.b);
        xb = df::fast_two_sum(xb.hi, xb.lo + C.lb);
      }
      if (act0) {
        svb = df::add(svb, df::mul(Vka, xa));
        sv = df::add(sv, Vka);
      }
      if (act1) {
        svb = df::add(svb, df::mul(Vkb, xb));
        sv = df::add(sv, Vkb);
      }
    }
    const float2 wpzk = wpz[k], wmzk = wmz[k];
    if (CYL) {
      wpy = a.wy[k];
      wmy = wpy;
    }
    // point a: east (the pair's inner face), west, south, north, up, down
    const Diff dab = diff_of<FAST>(C.b, C.a);
    const Diff dua = diff_of<FAST>(P.a, C.a), dub = diff_of<FAST>(P.b, C.b);
    flux_of<FAST>(Sa, wpxa, dab);
    flux_of<FAST>(Sa, wmxa, diff_of<FAST>(wa, C.a));
    flux_of<FAST>(Sa, wmy, diff_of<FAST>(S.a, C.a));
    flux_of<FAST>(Sa, wpy, diff_of<FAST>(N.a, C.a));
    flux_of<FAST>(Sa, wpzk, dua);
    flux_of<FAST>(Sa, wmzk, dza);
    // point b
    flux_of<FAST>(Sb, wpxb, diff_of<FAST>(eb, C.b));
    flux_of<FAST>(Sb, wmxb, neg(dab));
    flux_of<FAST>(Sb, wmy, diff_of<FAST>(S.b, C.b));
    flux_of<FAST>(Sb, wpy, diff_of<FAST>(N.b, C.b));
    flux_of<FAST>(Sb, wpzk, dub);
    flux_of<FAST>(Sb, wmzk, dzb);
    float sla = 0.f, slb = 0.f;  // lambda L applied to the low parts, FP32
    if (MODE == 1 && LO) {
      sla = fmaf(wpxa.x, C.lb - C.la, sla);
      sla = fmaf(wmxa.x, wal - C.la, sla);
      sla = fmaf(wmy.x, S.la - C.la, sla);
      sla = fmaf(wpy.x, N.la - C.la, sla);
      sla = fmaf(wpzk.x, P.la - C.la, sla);
      sla = fmaf(wmzk.x, mla - C.la, sla);
      slb = fmaf(wpxb.x, ebl - C.lb, slb);
      slb = fmaf(wmxb.x, C.la - C.lb, slb);
      slb = fmaf(wmy.x, S.lb - C.lb, slb);
      slb = fmaf(wpy.x, N.lb - C.lb, slb);
      slb = fmaf(wpzk.x, P.lb - C.lb, slb);
      slb = fmaf(wmzk.x, mlb - C.lb, slb);
    }
    const float2 w0k = w0z[k];
    if (wall_xy || w0k.x != 0.f) {  // wall term: only next to a Dirichlet wall
      const df::F2 wyz = df::add(df::make(w0y.x, w0y.y), df::make(w0k.x, w0k.y));
      const df::F2 ta = df::mul(df::add(df::make(w0xa.x, w0xa.y), wyz), df::make(C.a, C.la));
      const df::F2 tb = df::mul(df::add(df::make(w0xb.x, w0xb.y), wyz), df::make(C.b, C.lb));
      add_of<FAST>(Sa, ta.hi, ta.lo);
      add_of<FAST>(Sb, tb.hi, tb.lo);
    }
    if (SIG == 1) {
      add_of<FAST>(Sa, -C.a, -C.la);
      add_of<FAST>(Sb, -C.b, -C.lb);
    } else if (SIG == 2) {
      const df::F2 sg = df::make(a.sigma.x, a.sigma.y);
      const df::F2 ta = df::mul(sg, df::make(C.a, C.la));
      const df::F2 tb = df::mul(sg, df::make(C.b, C.lb));
      add_of<FAST>(Sa, -ta.hi, -ta.lo);
      add_of<FAST>(Sb, -tb.hi, -tb.lo);
    }
    // S.h + S.l: the rounding errors in S.l may exceed the cancelled S.h, so
    // the pair is rounded with a full two-sum
    const df::F2 ra = FAST ? df::make(Sa.h + (Sa.l + sla), 0.f) : df::two_sum(Sa.h, Sa.l + sla);
    const df::F2 rb = FAST ? df::make(Sb.h + (Sb.l + slb), 0.f) : df::two_sum(Sb.h, Sb.l + slb);
    // stores: the pair at once where both points exist
    {
      double oa = 0.0, ob = 0.0;
      if (OUT) {
        // every lane of the warp runs this (f2d_warp votes)
        oa = df::f2d_warp(h0) + (LO ? df::f2d_warp(C.a) + df::f2d_warp(C.la) : df::f2d_warp(C.a));
        ob = df::f2d_warp(h1) + (LO ? df::f2d_warp(C.b) + df::f2d_warp(C.lb) : df::f2d_warp(C.b));
      }
      if (VEC && act0) {  // VEC: act0 implies act1
        *reinterpret_cast<float2*>(rc + rk) = make_float2(ra.hi, rb.hi);
        if (MODE == 0) *reinterpret_cast<float2*>(rlc + rk) = make_float2(ra.lo, rb.lo);
        if (OUT) *reinterpret_cast<double2*>(outc + ok) = make_double2(oa, ob);
      } else if (!VEC) {
        if (act0) {
          rc[rk] = ra.hi;
          if (MODE == 0) rlc[rk] = ra.lo;
          if (OUT) outc[ok] = oa;
        }
        if (act1) {
          rc[rk + 1] = rb.hi;
          if (MODE == 0) rlc[rk + 1] = rb.lo;
          if (OUT) outc[ok + 1] = ob;
        }
      }
    }
    if (act0) {
      srr = fmaf(ra.hi, ra.hi, srr);
      if (MODE == 0) sbb = MEAN ? fmaf(ba.hi + mean_h, ba.hi + mean_h, sbb) : fmaf(ba.hi, ba.hi, sbb);
      rmax = fmaxf(rmax, fabsf(ra.hi));
    }
    if (act1) {
      srr = fmaf(rb.hi, rb.hi, srr);
      if (MODE == 0) sbb = MEAN ? fmaf(bb.hi + mean_h, bb.hi + mean_h, sbb) : fmaf(bb.hi, bb.hi, sbb);
      rmax = fmaxf(rmax, fabsf(rb.hi));
    }
    dza = neg(dua);
    dzb = neg(dub);
    mla = C.la;
    mlb = C.lb;
    C = P;
    P = P2;
    S = S2;
    N = N2;
    E = E2;
    El = E2l;
    b0 = b02;
    b1 = b12;
    Q = Q2;
    h0 = h02;
    h1 = h12;
    ok += szi;
    rk += rsi;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    srr += __shfl_down_sync(0xffffffffu, srr, o);
    sbb += __shfl_down_sync(0xffffffffu, sbb, o);
    rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    if (MEAN) {
      svb = df::add(svb, df::make(__shfl_down_sync(0xffffffffu, svb.hi, o), __shfl_down_sync(0xffffffffu, svb.lo, o)));
      sv = df::add(sv, df::make(__shfl_down_sync(0xffffffffu, sv.hi, o), __shfl_down_sync(0xffffffffu, sv.lo, o)));
    }
  }
  if (lane == 0) {
    sh[4 * wy + 0] = (double)srr;
    sh[4 * wy + 1] = (double)sbb;
    sh[4 * wy + 2] = MEAN ? df::to_f64(svb) : 0.0;
    sh[4 * wy + 3] = MEAN ? df::to_f64(sv) : 0.0;
    if (rmax > 0.f) atomicMax(reinterpret_cast<unsigned int*>(a.rmax), __float_as_uint(rmax));
  }
  __syncthreads();
  if (lane == 0 && wy == 0) {
    double t[4] = {0, 0, 0, 0};
    for (int q = 0; q < kResTY; ++q)
      for (int c = 0; c < 4; ++c) t[c] += sh[4 * q + c];
    for (int c = 0; c < 4; ++c) a.partials[4 * bid + c] = t[c];
  }
}


// Residual grid: 64 x 8 columns per block (x pairs), `zchunk` planes marched
// per block.  Long marches amortise the loads of the planes above and below;
// grids with fewer blocks than SMs halve the march (down to 4 planes) until
// every SM has a block.  (Filling the SMs several times over made a lone
// small solve a little faster but concurrent small solves slower.)  The order
// of the reduction is fixed by the grid, which depends on the shape only.
dim3 resid_grid(int nx, int ny, int nz, int* zchunk) {
  const long long cols = (long long)((nx + kResBX - 1) / kResBX) * ((ny + kResTY - 1) / kResTY);
  int zc = kResZChunk;
  while (zc > 4 && cols * ((nz + zc - 1) / zc) < 152) zc /= 2;
  *zchunk = zc;
  return dim3((unsigned)((nx + kResBX - 1) / kResBX), (unsigned)((ny + kResTY - 1) / kResTY),
              (unsigned)((nz + zc - 1) / zc));
}

// Final reduction of the per-block partials (fixed order: deterministic) and
// the convergence bookkeeping, by one block of nt threads (t = thread index).
// kind 0: initial pass (b only): record ||b||^2 and the volume-weighted mean
// kind 1: first residual check; kind 2: later check (counts a refinement step)
__device__ void finish_block(const double* __restrict__ partials, int nblocks, DevStatus* st, double tol, int kind,
                             int want_mean, int t, int nt) {
  __shared__ double shf[4 * 32];
  double s[4] = {0, 0, 0, 0};
  // 8 partial records per thread in flight (16-byte loads), fixed order
  const double2* p2 = reinterpret_cast<const double2*>(partials);
  for (int q0 = t; q0 < nblocks; q0 += 8 * nt) {
    double2 v[8][2];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = q0 + u * nt;
      if (q < nblocks) {
        v[u][0] = p2[2 * q];
        v[u][1] = p2[2 * q + 1];
      } else {
        v[u][0] = v[u][1] = make_double2(0.0, 0.0);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      s[0] += v[u][0].x;
      s[1] += v[u][0].y;
      s[2] += v[u][1].x;
      s[3] += v[u][1].y;
    }
  }
  for (int o = 16; o > 0; o >>= 1)
    for (int c = 0; c < 4; ++c) s[c] += __shfl_down_sync(0xffffffffu, s[c], o);
  const int w = t / 32, ln = t % 32;
  if (ln == 0)
    for (int c = 0; c < 4; ++c) shf[4 * w + c] = s[c];
  __syncthreads();
  if (t != 0) return;
  double tt[4] = {0, 0, 0, 0};
  for (int q = 0; q < nt / 32; ++q)
    for (int c = 0; c < 4; ++c) tt[c] += shf[4 * q + c];
  if (kind == 0) {
    // the solve's status starts here (no kernel of the solve reads it before)
    st->tol_used = tol;
    st->refine_steps = 0;
    st->iters = 0;
    st->error = 0;
    st->bnorm2 = tt[1];
    if (want_mean) st->mean_b = tt[2] / tt[3];
    st->rel_res = 1.0;
    st->done = 0;
    if (!isfinite(tt[1])) {  // non-finite right-hand side: nothing more runs
      st->error = 7;
      st->done = 1;
    }
    return;
  }
  if (st->error == 7) {  // a non-finite right-hand side stays reported as such
    st->done = 1;
    return;
  }
  // the first check (r_1 = b - A H) also measures ||b||; later checks reuse it
  const double bn2 = kind == 1 ? tt[1] : st->bnorm2;
  const double rel = bn2 > 0.0 ? sqrt(tt[0] / bn2) : sqrt(tt[0]);
  if (kind == 1) {
    st->refine_steps = 0;
    st->scal[1] = rel;  // ||r_1|| / ||b||: bounds the FP32 correction residual's error
  } else {
    st->refine_steps += 1;
  }
  if (want_mean) st->scal[0] = tt[2] / tt[3];  // volume-weighted mean of the current solution
  st->rel_res = rel;
  st->bnorm2 = bn2;
  if (!isfinite(rel)) {
    st->error = 1;
    st->done = 1;
  } else {
    st->done = rel <= tol ? 1 : 0;
  }
}


}  // namespace
}  // namespace fdi
