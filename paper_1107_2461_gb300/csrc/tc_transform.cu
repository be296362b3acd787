// Split-precision eigenvector transform on the tcgen05 tensor cores.
//
// One pass of the tensor-product solver (Sec. 3, Eq. 25/29) applies a dense
// n x n matrix T (E_d^{-1} forward, E_d back) along one direction of a field:
//     out(r, k) = sum_j T[k][j] in(r, j)       for every row r of the field.
// This is a GEMM with M = rows (128 per tile), N = n outputs and K = n; it is
// run in mixed precision: every operand x is scaled by a power of two and
// split into two fp16 parts, x = hi + lo, and the three products
//     A_hi*B_hi + A_hi*B_lo + A_lo*B_hi
// are accumulated in FP32 in tensor memory (about 22 significant bits of each
// operand; the refinement loop around the solver restores FP64 accuracy).
//
// Data layout: the input field is a row-major [R][pitch] FP32 matrix with the
// contraction index contiguous; the pass sequence of the solver writes each
// intermediate field in the orientation the next pass reads (see mixed.cu).
// The transform matrix T is split at plan time into B = [T_hi; T_lo] fp16
// [2*N_pad][K_pad] (row k scaled by its own power of two, undone per output
// column in the epilogue) and streamed by TMA.
//
// Warp roles of the persistent CTA (one per SM, 480 threads):
//   warp 0      TMA producer of the B chunks (each CTA loads its own copy; L2-resident)
//   warp 1      TMEM allocator and single-thread MMA issuer
//   warps 2-9   converters: read FP32 rows of A from shared memory, scale,
//               split to fp16 hi/lo, store them in the 64-byte swizzled
//               K-major layout of the MMA stage
//   warps 10-13 epilogue: TMEM -> registers -> unscale -> global store
//   warp 14     TMA producer of the FP32 A chunks (128 rows x 32 columns)
// Three MMA stages of K = 32, three FP32 A slots ahead of them (48 KB of input
// in flight per SM), two TMEM accumulators of N_pad columns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "fdi_internal.h"
#include "tc_common.cuh"
#include "tc_transform.h"

namespace fdi {
namespace {

constexpr int BM = 128;
constexpr int BK = 32;                       // fp16 K per chunk: 64-byte rows, 64-byte swizzle
constexpr int STAGES = 3;
constexpr int NA32 = 3;                      // FP32 A slots (TMA, 128-byte swizzle)
constexpr int NMAX = 256;
constexpr int ROWB = BK * 2;                 // bytes per operand row in a stage
constexpr int A_BYTES = BM * ROWB;           // one fp16 half of an A chunk: 8 KB
constexpr int B_BYTES = NMAX * ROWB;         // one fp16 half of a B chunk: up to 16 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int A32_BYTES = BM * BK * 4;      // 16 KB
constexpr int NCONV = 8;
constexpr int WARP_A = 2 + NCONV + 4;         // A producer warp
constexpr int THREADS = 32 * (WARP_A + 1);
constexpr bool kTmaTransposed = false;
constexpr int EPI_WARP_BYTES = 8 * 1024;      // per epilogue warp: transpose tile (32 x 33) or two TMA staging tiles (32 x 32)
constexpr int TP_BYTES = 4 * EPI_WARP_BYTES;
constexpr int BAR_BYTES = 256;
constexpr int CS_BYTES = NMAX * 4;            // per-column unscale factors
constexpr int A32_OFF = STAGES * STAGE_BYTES;
constexpr int EPI_OFF = A32_OFF + NA32 * A32_BYTES;  // 1024-byte aligned
constexpr int BAR_OFF = EPI_OFF + TP_BYTES;
// the dynamic block starts 1024-byte aligned (the static block is padded to
// 1024 bytes by the alignment of the extern declaration; checked at run time)
constexpr int SMEM_BYTES = BAR_OFF + BAR_BYTES + CS_BYTES;
static_assert(SMEM_BYTES + 1024 <= 232448, "shared memory budget");

__device__ __forceinline__ float scale_from_max(float mx) {
  // power of two that maps mx into [2^14, 2^15): fp16 keeps 11 bits there and
  // the split low part stays a normal number for values down to mx * 2^-17
  uint32_t b = __float_as_uint(mx);
  int e = (int)((b >> 23) & 0xff);
  if (e == 0 || e == 255) return 1.0f;
  int se = 127 + 14 - (e - 127);
  se = se < 1 ? 1 : (se > 254 ? 254 : se);
  return __uint_as_float((uint32_t)se << 23);
}


__global__ void __launch_bounds__(THREADS, 1)
    k_tc_transform(const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmA,
                   const __grid_constant__ CUtensorMap tmO, TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // the swizzled layouts need a 1024-byte aligned base; the launch reserves no
  // slack for re-alignment, so a misaligned block reports an error instead
  if ((tc::smem_u32(smem_raw) & 1023u) != 0u) {
    pdl_wait();
    if (threadIdx.x == 0) atomicExch(a.err, 7);
    return;
  }
  uint8_t* smem = smem_raw;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + BAR_OFF);
  uint64_t* full_b = bars;                  // B chunk landed (TMA transaction bytes)
  uint64_t* conv = bars + STAGES;           // A chunk converted (NCONV warp arrivals)
  uint64_t* empty = bars + 2 * STAGES;      // stage consumed by the MMAs (one commit)
  uint64_t* accf = bars + 3 * STAGES;       // accumulator complete
  uint64_t* acce = bars + 3 * STAGES + 2;   // accumulator drained by the epilogue
  uint64_t* a_full = bars + 3 * STAGES + 4;          // FP32 A chunk landed (TMA bytes)
  uint64_t* a_empty = bars + 3 * STAGES + 4 + NA32;  // FP32 A chunk read (NCONV warp arrivals)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * STAGES + 4 + 2 * NA32);
  uint64_t* mma_drain = bars + 3 * STAGES + 4 + 2 * NA32 + 1;  // MMAs issued before a failure completed
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const long long wl = a.wait_cycles > 0 ? a.wait_cycles : tc::kWaitCycles;
  const int N_pad = a.N_pad;
  uint32_t tmem_cols = 32;
  while (tmem_cols < (uint32_t)(2 * N_pad)) tmem_cols <<= 1;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(&full_b[s], 1);
      tc::mbar_init(&conv[s], NCONV);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&accf[b], 1);
      tc::mbar_init(&acce[b], 4);
    }
    for (int b = 0; b < NA32; ++b) {
      tc::mbar_init(&a_full[b], 1);
      tc::mbar_init(&a_empty[b], NCONV);
    }
    tc::mbar_init(mma_drain, 1);
    s_abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0 && lane == 0) tc::prefetch_tmap(&tmB);
  if (warp == WARP_A && lane == 0) tc::prefetch_tmap(&tmA);
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, tmem_cols);
    tc::tmem_relinquish();
  }
  // per output column: the matrix row's scale (plan data), times the input's
  // inverse scale below (both powers of two)
  float* s_cs = reinterpret_cast<float*>(smem + BAR_OFF + BAR_BYTES);
  float csk[(NMAX + THREADS - 1) / THREADS];
#pragma unroll
  for (int q = 0; q < (NMAX + THREADS - 1) / THREADS; ++q) {
    const int k = threadIdx.x + q * THREADS;
    csk[q] = k < N_pad ? a.col_scale[k] : 0.f;
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // Everything above touches no data of the previous kernel in the stream, so
  // under programmatic dependent launch it overlaps that kernel's tail; from
  // here on the previous kernel has completed and its writes are visible.
  pdl_wait();
  const int skip = a.skip ? *a.skip : 0;  // the same for every thread
  const float in_scale = a.scale_in ? *a.scale_in : 1.0f;
  if (skip) {
    if (warp == 1) tc::tmem_dealloc(tmem_base, tmem_cols);
    return;
  }
  {
    const float inv_s = 1.0f / scale_from_max(in_scale);
#pragma unroll
    for (int q = 0; q < (NMAX + THREADS - 1) / THREADS; ++q) {
      const int k = threadIdx.x + q * THREADS;
      if (k < N_pad) s_cs[k] = csk[q] * inv_s;
    }
  }
  __syncthreads();

  const long long num_tiles = (a.R + BM - 1) / BM;
  // work items: tiles below n_full whole, the tail's tiles as two halves
  // (columns [0, N_pad / 2) and [N_pad / 2, N_pad)); every role walks the same
  // items in the same order
  const long long n_full = (a.n_full > 0 && a.n_full < num_tiles) ? a.n_full : num_tiles;
  const long long num_items = n_full + 2 * (num_tiles - n_full);
  const long long my_iters = blockIdx.x < num_items ? (num_items - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  // item `it` of this CTA: its tile, and half = -1 (whole), 0 or 1
  auto item_tile = [&](long long it, int* half) -> long long {
    const long long item = blockIdx.x + it * gridDim.x;
    if (item < n_full) {
      *half = -1;
      return item;
    }
    const long long h = item - n_full;
    *half = (int)(h & 1);
    return n_full + (h >> 1);
  };
  const int nK = a.nK;

  if (warp == 0) {
    // ---------------- TMA producer (B) ----------------
    if (lane == 0) {
      const uint32_t bbytes = (uint32_t)(2 * N_pad * ROWB);
      uint32_t g = 0;
      for (long long it = 0; it < my_iters && !s_abort; ++it) {
        for (int kc = 0; kc < nK; ++kc, ++g) {
          const int s = g % STAGES;
          const uint32_t ph = (g / STAGES) & 1;
          if (!tc::mbar_wait(&empty[s], ph ^ 1, &s_abort, wl)) {
            s_abort = 1;
            atomicExch(a.err, 1);
            break;
          }
          tc::mbar_expect_tx(&full_b[s], bbytes);
          uint8_t* st = smem + s * STAGE_BYTES;
          tc::tma_load_2d(tc::smem_u32(st + 2 * A_BYTES), &tmB, kc * BK, 0, &full_b[s]);
          tc::tma_load_2d(tc::smem_u32(st + 2 * A_BYTES + B_BYTES), &tmB, kc * BK, N_pad, &full_b[s]);
        }
      }
      // the last STAGES loads issued may still be writing shared memory (after
      // a failure nobody consumes them); their phases complete regardless, and
      // a consumed one has completed already
      for (uint32_t g2 = g > STAGES ? g - STAGES : 0; g2 < g; ++g2)
        tc::mbar_drain(&full_b[g2 % STAGES], (g2 / STAGES) & 1);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      uint32_t g = 0;
      for (long long it = 0; it < my_iters && !s_abort; ++it) {
        int half = -1;
        item_tile(it, &half);
        // a half item accumulates its columns where the whole tile would
        const uint32_t coff = half == 1 ? (uint32_t)(N_pad / 2) : 0u;
        const uint32_t idesc = tc::idesc_f16_f32(BM, half < 0 ? N_pad : N_pad / 2);
        const int buf = (int)(it & 1);
        const uint32_t aph = (uint32_t)((it >> 1) & 1);
        if (!tc::mbar_wait(&acce[buf], aph ^ 1, &s_abort, wl)) {
          s_abort = 1;
          atomicExch(a.err, 2);
          break;
        }
        tc::tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(buf * N_pad) + coff;
        bool ok = true;
        for (int kc = 0; kc < nK; ++kc, ++g) {
          const int s = g % STAGES;
          const uint32_t ph = (g / STAGES) & 1;
          if (!tc::mbar_wait(&full_b[s], ph, &s_abort, wl) || !tc::mbar_wait(&conv[s], ph, &s_abort, wl)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          uint8_t* st = smem + s * STAGE_BYTES;
          const uint32_t ahi = tc::smem_u32(st), alo = tc::smem_u32(st + A_BYTES);
          const uint32_t bhi = tc::smem_u32(st + 2 * A_BYTES) + coff * ROWB;
          const uint32_t blo = tc::smem_u32(st + 2 * A_BYTES + B_BYTES) + coff * ROWB;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            const uint32_t off = kk * 32;
            const uint32_t acc = (kc > 0 || kk > 0) ? 1u : 0u;
            tc::mma_f16(d, tc::sdesc_k_sw64(ahi + off), tc::sdesc_k_sw64(bhi + off), idesc, acc);
            tc::mma_f16(d, tc::sdesc_k_sw64(ahi + off), tc::sdesc_k_sw64(blo + off), idesc, 1u);
            tc::mma_f16(d, tc::sdesc_k_sw64(alo + off), tc::sdesc_k_sw64(bhi + off), idesc, 1u);
          }
          tc::mma_commit(&empty[s]);
        }
        if (!ok) {
          s_abort = 1;
          atomicExch(a.err, 3);
          break;
        }
        tc::mma_commit(&accf[buf]);
      }
      // every MMA issued has completed before TMEM and the stages are released
      // (also when another role gave up waiting for them)
      tc::mma_commit(mma_drain);
      tc::mbar_drain(mma_drain, 0);
    }
  } else if (warp < 2 + NCONV) {
    // ---------------- converters ----------------
    // Each thread owns 2 (row, 32-byte) slots of a 128 x 32 A chunk: it reads
    // the FP32 values from the TMA slot (128-byte swizzle: 16-byte unit u of
    // row r sits at unit u ^ (r & 7), conflict free), scales, splits and stores
    // 16 fp16 hi and lo values into the MMA stage.
    const int ct = (warp - 2) * 32 + lane;  // 0..255
    const float sA = scale_from_max(in_scale);
    const int c8 = ct & 3;                  // 32-byte group within the 128-byte row
    // the two (row, 8-wide k group) pieces this thread converts per chunk:
    // K-major slots: rows ct/4 and ct/4 + 64, k group c8; MN-major slots: row
    // ct % 128, k groups 2 (ct / 128) and 2 (ct / 128) + 1
    const bool a_mn = a.a_mn != 0;
    const int row_q[2] = {a_mn ? (ct & 127) : (ct >> 2), a_mn ? (ct & 127) : (ct >> 2) + 64};
    const int kofs_q[2] = {a_mn ? (ct >> 7) * 16 : c8 * 8, a_mn ? (ct >> 7) * 16 + 8 : c8 * 8};
    const long long total = my_iters * nK;
    int kc = 0;
    for (long long gi = 0; gi < total && !s_abort; ++gi) {
      const uint32_t g = (uint32_t)gi;
      const int sa = g % NA32;
      const uint32_t pa = (g / NA32) & 1;
      const int s = g % STAGES;
      const uint32_t ph = (g / STAGES) & 1;
      if (!tc::mbar_wait(&a_full[sa], pa, &s_abort, wl)) {
        atomicExch(a.err, 4);
        break;
      }
      const uint8_t* src = smem + A32_OFF + sa * A32_BYTES;
      float v[2][8];
      if (!a_mn) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int row = row_q[q];
          const float4 x0 = *reinterpret_cast<const float4*>(src + row * 128 + (((2 * c8) ^ (row & 7)) << 4));
          const float4 x1 = *reinterpret_cast<const float4*>(src + row * 128 + (((2 * c8 + 1) ^ (row & 7)) << 4));
          v[q][0] = x0.x; v[q][1] = x0.y; v[q][2] = x0.z; v[q][3] = x0.w;
          v[q][4] = x1.x; v[q][5] = x1.y; v[q][6] = x1.z; v[q][7] = x1.w;
        }
      } else {
        // MN-major slot [32 k][128 m]: a warp reads 32 consecutive m of one k
        const float* sf = reinterpret_cast<const float*>(src);
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int e = 0; e < 8; ++e) v[q][e] = sf[(kofs_q[q] + e) * BM + row_q[q]];
      }
      if (!tc::mbar_wait(&empty[s], ph ^ 1, &s_abort, wl)) {
        atomicExch(a.err, 4);
        break;
      }
      uint8_t* st = smem + s * STAGE_BYTES;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int row = row_q[q];
        const int k0 = kc * BK + kofs_q[q];
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
          const float x0 = (k0 + e < a.K) ? v[q][e] * sA : 0.f;
          const float x1 = (k0 + e + 1 < a.K) ? v[q][e + 1] * sA : 0.f;
          // packed conversions (one instruction per pair, round to nearest)
          const __half2 h = __floats2half2_rn(x0, x1);
          const float2 hf = __half22float2(h);
          const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
          hw[e / 2] = *reinterpret_cast<const uint32_t*>(&h);
          lw[e / 2] = *reinterpret_cast<const uint32_t*>(&l);
        }
        const uint32_t off = tc::sw64_offset(row, kofs_q[q]);
        *reinterpret_cast<uint4*>(st + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4*>(st + A_BYTES + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      }
      // the FP32 values were consumed above: the slot may be refilled
      tc::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        tc::mbar_arrive(&a_empty[sa]);
        tc::mbar_arrive(&conv[s]);
      }
      if (++kc == nK) kc = 0;
    }
  } else if (warp == WARP_A) {
    // ---------------- TMA producer (FP32 A) ----------------
    if (lane == 0) {
      uint32_t g = 0;
      for (long long it = 0; it < my_iters && !s_abort; ++it) {
        int half = -1;
        const long long tile = item_tile(it, &half);
        const int row0 = (int)(tile * BM);
        for (int kc = 0; kc < nK; ++kc, ++g) {
          const int sa = g % NA32;
          const uint32_t pa = (g / NA32) & 1;
          if (!tc::mbar_wait(&a_empty[sa], pa ^ 1, &s_abort, wl)) {
            s_abort = 1;
            atomicExch(a.err, 6);
            break;
          }
          tc::mbar_expect_tx(&a_full[sa], (uint32_t)A32_BYTES);
          if (!a.a_mn) {
            tc::tma_load_2d(tc::smem_u32(smem + A32_OFF + sa * A32_BYTES), &tmA, kc * BK, row0, &a_full[sa]);
          } else {
            // MN-major input: box of 128 consecutive m (one slab) x 32 k rows
            const long long slab = (long long)row0 / a.a_mslab;
            tc::tma_load_2d(tc::smem_u32(smem + A32_OFF + sa * A32_BYTES), &tmA, (int)((long long)row0 % a.a_mslab),
                            (int)(slab * a.K + (long long)kc * BK), &a_full[sa]);
          }
        }
      }
      for (uint32_t g2 = g > NA32 ? g - NA32 : 0; g2 < g; ++g2)
        tc::mbar_drain(&a_full[g2 % NA32], (g2 / NA32) & 1);
    }
  } else {
    // ---------------- epilogue ----------------
    // Each thread holds one accumulator row (TMEM lane) and 32 columns per
    // load.  Every 32 x 32 block goes through a shared tile (stride 33: conflict
    // free both ways); after the transpose a lane owns 4 consecutive rows of one
    // column (transposed outputs) or 4 consecutive columns of one row (row-major
    // outputs) and stores them with one 16-byte access where the layout allows.
    const int q = warp & 3;  // TMEM lane quarter accessible to this warp
    float* tp0 = reinterpret_cast<float*>(smem + EPI_OFF + (warp - (2 + NCONV)) * EPI_WARP_BYTES);
    uint32_t nstore = 0;  // TMA stores issued by this warp: staging tile nstore & 1 is next
    const bool rowmajor = a.col_stride == 1;
    // vector stores need 16-byte aligned groups of 4 along the contiguous index
    const bool vec_t = !rowmajor && a.row_stride == 1 && (a.S % 4 == 0) && (a.slab_stride % 4 == 0) &&
                       (a.col_stride % 4 == 0);
    const bool vec_r = rowmajor && a.row_stride % 4 == 0 && a.slab_stride % 4 == 0 &&
                       (reinterpret_cast<uintptr_t>(a.out_f32) & 15u) == 0;
    const int g8 = lane >> 3, l8 = lane & 7;  // after the transpose: group of 8 lanes, lane in group
    float vmax = 0.f;
    for (long long it = 0; it < my_iters && !s_abort; ++it) {
      int half = -1;
      const long long tile = item_tile(it, &half);
      const int c_lo = half == 1 ? N_pad / 2 : 0, c_hi = half == 0 ? N_pad / 2 : N_pad;
      const int buf = (int)(it & 1);
      const uint32_t aph = (uint32_t)((it >> 1) & 1);
      if (!tc::mbar_wait(&accf[buf], aph, &s_abort, wl)) {
        atomicExch(a.err, 5);
        break;
      }
      tc::tc_fence_after();
      const long long wrow0 = tile * BM + 32 * q;  // first row of this warp
      const bool tvalid = tile < num_tiles;
      const int nrows = tvalid ? (int)max(0LL, min((long long)32, a.R - wrow0)) : 0;
      // output base of this lane's own row (row = wrow0 + lane)
      long long base = 0;
      {
        const long long row = wrow0 + lane;
        if (row < a.R) base = (row / a.S) * a.slab_stride + (row % a.S) * a.row_stride;
      }
      // bases of the 4 rows this lane stores after a transpose (transposed outputs)
      long long tb[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) tb[e] = __shfl_sync(0xffffffffu, base, 4 * l8 + e);
      for (int c0 = c_lo; c0 < c_hi; c0 += 32) {
        uint32_t r[32];
        tc::tmem_ld32(tmem_base + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * N_pad + c0), r);
        tc::tmem_ld_wait();
        if (a.tma_store) {
          // unscale into a staging tile and hand it to a TMA store; rows past
          // R and columns past n_out hold zeros (zero-filled A rows, zero B
          // rows) and are clipped by the store.  Two staging tiles alternate:
          // the store two back (same tile) must have read it, the last one may
          // still be reading the other
          float* tp = tp0 + (nstore & 1u) * 1024;
          if (lane == 0) tc::bulk_wait_read_1();
          __syncwarp();
          if (a.tma_store == 1) {
            // staging [column][row]: 32 rows of one column are 128 contiguous bytes
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const float v = __uint_as_float(r[j]) * s_cs[c0 + j];
              vmax = fmaxf(vmax, fabsf(v));
              tp[j * 32 + lane] = v;
            }
          } else {
            // staging [row][column] in the 128-byte swizzle (16-byte unit u of row
            // `lane` at unit u ^ (lane & 7))
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              float v4[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                v4[e] = __uint_as_float(r[4 * u + e]) * s_cs[c0 + 4 * u + e];
                vmax = fmaxf(vmax, fabsf(v4[e]));
              }
              *reinterpret_cast<float4*>(tp + lane * 32 + ((u ^ (lane & 7)) << 2)) =
                  make_float4(v4[0], v4[1], v4[2], v4[3]);
            }
          }
          tc::fence_proxy_async_smem();
          __syncwarp();
          if (nrows > 0) {
            if (lane == 0) {
              const uint32_t stg = tc::smem_u32(tp);  // 1024-byte aligned
              if (a.tma_store == 1)
                tc::tma_store_3d(&tmO, stg, (int)(wrow0 % a.S), c0, (int)(wrow0 / a.S));
              else
                tc::tma_store_2d(&tmO, stg, c0, (int)wrow0);
              tc::bulk_commit();
            }
            ++nstore;
          }
          continue;
        }
        float* tp = tp0;
#pragma unroll
        for (int j = 0; j < 32; ++j) tp[lane * 33 + j] = __uint_as_float(r[j]);
        __syncwarp();
        if (!rowmajor) {
          // lane -> column c0 + 4*qq + g8, rows 4*l8 .. 4*l8+3 of the warp block
          const int rr = 4 * l8;
#pragma unroll
          for (int qq = 0; qq < 8; ++qq) {
            const int cl = 4 * qq + g8;
            const int k = c0 + cl;
            if (k < a.n_out) {
              const float cs = s_cs[k];
              float v4[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                v4[e] = tp[(rr + e) * 33 + cl] * cs;
                if (rr + e < nrows) vmax = fmaxf(vmax, fabsf(v4[e]));
              }
              const long long koff = (long long)k * a.col_stride;
              if (vec_t && rr + 3 < nrows) {
                *reinterpret_cast<float4*>(a.out_f32 + tb[0] + koff) = make_float4(v4[0], v4[1], v4[2], v4[3]);
              } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                  if (rr + e < nrows) a.out_f32[tb[e] + koff] = v4[e];
              }
            }
          }
        } else {
          // lane -> row 4*qq + g8 of the warp block, columns c0 + 4*l8 .. +3
          const int cc = 4 * l8;
          float cs[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int k = c0 + cc + e;
            cs[e] = (k < a.n_out) ? s_cs[k] : 0.f;
          }
          const bool fullcols = c0 + cc + 3 < a.n_out;
          if (a.mode == TC_OUT_F32) {
#pragma unroll
            for (int qq = 0; qq < 8; ++qq) {
              const int rl = 4 * qq + g8;
              const long long brow = __shfl_sync(0xffffffffu, base, rl);
              if (rl < nrows) {
                float v4[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) v4[e] = tp[rl * 33 + cc + e] * cs[e];
                float* o = a.out_f32 + brow + c0 + cc;
                if (vec_r && fullcols) {
                  *reinterpret_cast<float4*>(o) = make_float4(v4[0], v4[1], v4[2], v4[3]);
                } else {
#pragma unroll
                  for (int e = 0; e < 4; ++e)
                    if (c0 + cc + e < a.n_out) o[e] = v4[e];
                }
#pragma unroll
                for (int e = 0; e < 4; ++e)
                  if (c0 + cc + e < a.n_out) vmax = fmaxf(vmax, fabsf(v4[e]));
              }
            }
          } else {
            // double-float accumulation into the (out_f32, out_lo) planes: rows in
            // groups of 4 with the loads of a group issued before any update
#pragma unroll
            for (int q4 = 0; q4 < 8; q4 += 4) {
              float oh[4][4], ol[4][4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int rl = 4 * (q4 + u) + g8;
                const long long brow = __shfl_sync(0xffffffffu, base, rl) + c0 + cc;
                if (rl < nrows && vec_r && fullcols) {
                  const float4 h = *reinterpret_cast<const float4*>(a.out_f32 + brow);
                  const float4 l = a.lo_valid ? *reinterpret_cast<const float4*>(a.out_lo + brow)
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
                  oh[u][0] = h.x; oh[u][1] = h.y; oh[u][2] = h.z; oh[u][3] = h.w;
                  ol[u][0] = l.x; ol[u][1] = l.y; ol[u][2] = l.z; ol[u][3] = l.w;
                } else {
#pragma unroll
                  for (int e = 0; e < 4; ++e) {
                    const bool ok = rl < nrows && c0 + cc + e < a.n_out;
                    oh[u][e] = ok ? a.out_f32[brow + e] : 0.f;
                    ol[u][e] = (ok && a.lo_valid) ? a.out_lo[brow + e] : 0.f;
                  }
                }
              }
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int rl = 4 * (q4 + u) + g8;
                const long long brow = __shfl_sync(0xffffffffu, base, rl) + c0 + cc;
                if (rl >= nrows) continue;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  // (oh, ol) + val: two-sum of the high parts, low parts added, fast renormalisation
                  const float val = tp[rl * 33 + cc + e] * cs[e];
                  const float sh = oh[u][e] + val;
                  const float bb = sh - oh[u][e];
                  const float er = (oh[u][e] - (sh - bb)) + (val - bb) + ol[u][e];
                  const float nh = sh + er;
                  oh[u][e] = nh;
                  ol[u][e] = er - (nh - sh);
                }
                if (vec_r && fullcols) {
                  *reinterpret_cast<float4*>(a.out_f32 + brow) = make_float4(oh[u][0], oh[u][1], oh[u][2], oh[u][3]);
                  *reinterpret_cast<float4*>(a.out_lo + brow) = make_float4(ol[u][0], ol[u][1], ol[u][2], ol[u][3]);
                } else {
#pragma unroll
                  for (int e = 0; e < 4; ++e)
                    if (c0 + cc + e < a.n_out) {
                      a.out_f32[brow + e] = oh[u][e];
                      a.out_lo[brow + e] = ol[u][e];
                    }
                }
              }
            }
          }
        }
        __syncwarp();
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&acce[buf]);
    }
    if (a.tma_store && lane == 0) tc::bulk_wait_all();
    if (a.scale_out) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
      if (lane == 0 && vmax > 0.f) atomicMax(reinterpret_cast<unsigned int*>(a.scale_out), __float_as_uint(vmax));
    }
  }

  tc::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem_base, tmem_cols);
  }
}

__global__ void k_prep_b(const double* __restrict__ T, int n, int N_pad, int K_pad, __half* __restrict__ B,
                         float* __restrict__ col_scale) {
  // row k of T (output k) -> scaled by a power of two, split into fp16 hi/lo
  const int k = blockIdx.x;
  __shared__ double smax[256];
  double mx = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    if (k < n) mx = fmax(mx, fabs(T[(size_t)k * n + j]));
  smax[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
    __syncthreads();
  }
  mx = smax[0];
  double sc = 1.0;
  if (mx > 0.0) sc = exp2(14.0 - floor(log2(mx)));
  if (threadIdx.x == 0) col_scale[k] = (float)(1.0 / sc);
  for (int j = threadIdx.x; j < K_pad; j += blockDim.x) {
    double t = (k < n && j < n) ? T[(size_t)k * n + j] * sc : 0.0;
    __half h = __double2half(t);
    __half l = __double2half(t - (double)__half2float(h));
    B[(size_t)k * K_pad + j] = h;
    B[(size_t)(N_pad + k) * K_pad + j] = l;
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

}  // namespace

fdi_status tc_prepare_matrix(fdi_plan* p, const double* T, int n, TcMatrix* m, cudaStream_t s) {
  m->n = n;
  m->N_pad = ((n + 31) / 32) * 32;
  m->K_pad = ((n + BK - 1) / BK) * BK;
  const size_t elems = (size_t)2 * m->N_pad * m->K_pad;
  FDI_CUDA_TRY(cudaMalloc(&m->B, elems * sizeof(__half)));
  FDI_CUDA_TRY(cudaMalloc(&m->col_scale, m->N_pad * sizeof(float)));
  FDI_CUDA_TRY(cudaMemsetAsync(m->col_scale, 0, m->N_pad * sizeof(float), s));
  k_prep_b<<<m->N_pad, 256, 0, s>>>(T, n, m->N_pad, m->K_pad, (__half*)m->B, m->col_scale);
  FDI_LAUNCH_CHECK(p);
  auto enc = encode_fn();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled entry point unavailable");
    return FDI_ERR_CUDA;
  }
  {
    // B chunks: N_pad rows x 32 fp16 (one half, hi or lo, of a stage's B operand)
    cuuint64_t dims[2] = {(cuuint64_t)m->K_pad, (cuuint64_t)(2 * m->N_pad)};
    cuuint64_t strides[1] = {(cuuint64_t)m->K_pad * sizeof(__half)};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)m->N_pad};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(reinterpret_cast<CUtensorMap*>(m->tmap), CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, m->B, dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      set_error("cuTensorMapEncodeTiled failed for a transform matrix");
      return FDI_ERR_CUDA;
    }
  }
  return FDI_OK;
}

// The matrix as the resident solve's MMA reads it from shared memory: for
// every K chunk of 32, the hi rows then the lo rows (N_pad each), every row 64
// bytes in the 64-byte swizzle layout; copied into shared memory as it is.
__global__ void k_res_image(const __half* __restrict__ B, int N_pad, int K_pad, uint8_t* __restrict__ img) {
  const int half = blockIdx.y, n = blockIdx.x;
  for (int k = threadIdx.x; k < K_pad; k += blockDim.x) {
    const size_t off = (size_t)(k / BK) * (2 * N_pad * ROWB) + (size_t)half * N_pad * ROWB + tc::sw64_offset(n, k % BK);
    *reinterpret_cast<__half*>(img + off) = B[((size_t)half * N_pad + n) * K_pad + k];
  }
}

fdi_status tc_resident_image(fdi_plan* p, const TcMatrix& m, uint8_t** img, cudaStream_t s) {
  const size_t bytes = (size_t)(m.K_pad / BK) * 2 * m.N_pad * ROWB;
  FDI_CUDA_TRY(cudaMalloc(img, bytes));
  k_res_image<<<dim3((unsigned)m.N_pad, 2), 128, 0, s>>>((const __half*)m.B, m.N_pad, m.K_pad, *img);
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

void tc_free_matrix(TcMatrix* m) {
  if (m->B) cudaFree(m->B);
  if (m->col_scale) cudaFree(m->col_scale);
  m->B = nullptr;
  m->col_scale = nullptr;
}

fdi_status launch_kernel(fdi_plan* p, const TcMatrix& m, const CUtensorMap& mapA, const CUtensorMap& mapO,
                         const TcArgs& args, long long tiles, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    FDI_CUDA_TRY(cudaFuncSetAttribute(k_tc_transform, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    attr_set = true;
  }
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  const long long grid = tiles < sms ? tiles : sms;
  // a partial last wave of tiles runs as half-width items spread over twice
  // as many CTAs (halves stay multiples of 32 columns)
  TcArgs a2 = args;
  a2.n_full = tiles;
  if (tiles > grid && m.N_pad % 64 == 0) {
    const long long tail = tiles % grid;
    if (tail > 0 && 2 * tail <= grid) a2.n_full = tiles - tail;
  }
  CUtensorMap map;
  memcpy(&map, m.tmap, sizeof(CUtensorMap));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(THREADS);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = args.pdl ? 1 : 0;
  FDI_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_tc_transform, map, mapA, mapO, a2));
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

fdi_status launch_tc_transform(fdi_plan* p, const TcMatrix& m, TcArgs args, const char* name, cudaStream_t s) {
  FDI_KTIMER(p, name, s);
  args.N_pad = m.N_pad;
  args.nK = (args.K + BK - 1) / BK;
  args.wait_cycles = p->wait_cycles;
  args.col_scale = m.col_scale;
  const long long tiles = (args.R + BM - 1) / BM;
  if (args.R > 0x7fffffffLL - BM || args.in_pitch % 4 != 0 || (reinterpret_cast<uintptr_t>(args.in) & 15u) != 0) {
    set_error("transform input must be 16-byte aligned with a pitch multiple of 4 and fewer than 2^31 rows");
    return FDI_ERR_INVALID_ARG;
  }
  // FP32 input rows as a 2D tensor [R][in_pitch]; 32 x 128 boxes, 128-byte swizzle;
  // rows past R and columns past the pitch read as zero
  auto enc = encode_fn();
  if (!enc) {
    set_error("cuTensorMapEncodeTiled entry point unavailable");
    return FDI_ERR_CUDA;
  }
  CUtensorMap mapA;
  // MN-major slabs hold whole 128-row tiles, or there is one slab as wide as
  // the tensor row (a ragged last tile then reads the zero fill past its end)
  const bool one_slab = args.a_mslab == args.R && args.a_mslab == args.in_pitch;
  if (args.a_mn && ((args.a_mslab % BM != 0 && !one_slab) || args.R % args.a_mslab != 0 ||
                    args.a_mslab > args.in_pitch || args.a_rows < (args.R / args.a_mslab) * (long long)args.K ||
                    args.a_rows > 0x7fffffffLL)) {
    set_error("MN-major transform input: slabs must hold whole 128-row tiles");
    return FDI_ERR_INVALID_ARG;
  }
  {
    // K-major: rows of K contiguous values, 32 x 128 boxes, 128-byte swizzle.
    // MN-major: a_rows rows of in_pitch values (m contiguous), 128 x 32 boxes.
    cuuint64_t dims[2] = {(cuuint64_t)args.in_pitch, (cuuint64_t)(args.a_mn ? args.a_rows : args.R)};
    cuuint64_t strides[1] = {(cuuint64_t)args.in_pitch * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)(args.a_mn ? BM : BK), (cuuint32_t)(args.a_mn ? BK : BM)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&mapA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(args.in), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, args.a_mn ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      set_error("cuTensorMapEncodeTiled failed for a transform input");
      return FDI_ERR_CUDA;
    }
  }
  // output through TMA stores where the layout allows: 16-byte aligned base and
  // strides, and (transposed outputs) slabs made of whole 32-row warp blocks
  CUtensorMap mapO;
  memset(&mapO, 0, sizeof(mapO));
  args.tma_store = 0;
  const bool out_aligned = (reinterpret_cast<uintptr_t>(args.out_f32) & 15u) == 0;
  if (args.mode == TC_OUT_F32 && out_aligned && args.n_out > 0) {
    cuuint32_t estr[3] = {1, 1, 1};
    // transposed outputs keep the thread stores (16-byte row groups after an
    // in-shared transpose), which measured faster than 32 x 32 TMA boxes of
    // 128-byte column segments; kTmaTransposed enables the TMA variant
    if (kTmaTransposed && args.row_stride == 1 && args.S % 32 == 0 && args.R % args.S == 0 &&
        args.col_stride % 4 == 0 && args.slab_stride % 4 == 0 && args.R / args.S < 0x7fffffffLL) {
      cuuint64_t dims[3] = {(cuuint64_t)args.S, (cuuint64_t)args.n_out, (cuuint64_t)(args.R / args.S)};
      cuuint64_t strides[2] = {(cuuint64_t)args.col_stride * sizeof(float), (cuuint64_t)args.slab_stride * sizeof(float)};
      cuuint32_t box[3] = {32, 32, 1};
      if (enc(&mapO, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, args.out_f32, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
        args.tma_store = 1;
    } else if (args.col_stride == 1 && args.S == args.R && args.row_stride % 4 == 0 && args.row_stride >= args.n_out) {
      cuuint64_t dims[2] = {(cuuint64_t)args.n_out, (cuuint64_t)args.R};
      cuuint64_t strides[1] = {(cuuint64_t)args.row_stride * sizeof(float)};
      cuuint32_t box[2] = {32, 32};
      if (enc(&mapO, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, args.out_f32, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
        args.tma_store = 2;
    }
  }
  return launch_kernel(p, m, mapA, mapO, args, tiles, s);
}

}  // namespace fdi
