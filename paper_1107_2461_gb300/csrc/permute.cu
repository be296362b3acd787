// Thomas axis other than z for cell-field plans (Sec. 3: the Thomas sweep runs
// along one direction, the paper's choice being the direction with the most
// grid points).  A plan whose Thomas axis is x or y keeps its fields with that
// axis outermost: the internal grid is the external one with two axes swapped,
// every solve copies the right-hand side into that order, runs the z-Thomas
// solver on it and copies the solution back.  Both copies are plain FP64
// permutations (bandwidth bound, 16 bytes per point each).
//
//   Thomas along x: external [z][y][x] <-> internal [x][y][z]  (swap x and z)
//   Thomas along y: external [z][y][x] <-> internal [y][z][x]  (swap y and z)
#include <algorithm>

#include "fdi_internal.h"

namespace fdi {
namespace {

constexpr int kT = 32;  // transpose tile

// out[b][m][a] = in[a][m][b] for a < A, m < M, b < B (b contiguous in `in`,
// a contiguous in `out`): one 32 x 32 tile of the (a, b) plane of one m per
// block, through shared memory (stride 33: no bank conflicts either way)
__global__ void __launch_bounds__(kT * 8) k_swap_first_last(const double* __restrict__ in, double* __restrict__ out,
                                                           int A, int M, int B) {
  __shared__ double tile[kT][kT + 1];
  const int b0 = blockIdx.x * kT, a0 = blockIdx.y * kT, m = blockIdx.z;
  const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
  for (int r = ty; r < kT; r += 8) {
    const int a = a0 + r, b = b0 + tx;
    if (a < A && b < B) tile[r][tx] = in[((long long)a * M + m) * B + b];
  }
  __syncthreads();
#pragma unroll
  for (int r = ty; r < kT; r += 8) {
    const int b = b0 + r, a = a0 + tx;
    if (a < A && b < B) out[((long long)b * M + m) * A + a] = tile[tx][r];
  }
}

// out[b][a][:] = in[a][b][:] for rows of R contiguous values
__global__ void k_swap_outer(const double* __restrict__ in, double* __restrict__ out, int A, int B, int R) {
  const long long rows = (long long)A * B;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const int a = (int)(row / B), b = (int)(row % B);
    const double* src = in + row * R;
    double* dst = out + ((long long)b * A + a) * R;
    for (int x = threadIdx.x; x < R; x += blockDim.x) dst[x] = src[x];
  }
}

}  // namespace

// external-order field `in` (n_ext = external cells) -> internal order (to_internal)
// or back; `axis` is the external Thomas axis (0 or 1)
fdi_status launch_axis_permute(fdi_plan* p, const double* in, double* out, bool to_internal, cudaStream_t s) {
  const int nx = p->n_ext[0], ny = p->n_ext[1], nz = p->n_ext[2];
  if (p->thomas_ext == 0) {
    // external [z][y][x] <-> internal [x][y][z]
    const int A = to_internal ? nz : nx, B = to_internal ? nx : nz;
    const dim3 grid((unsigned)((B + kT - 1) / kT), (unsigned)((A + kT - 1) / kT), (unsigned)ny);
    k_swap_first_last<<<grid, dim3(kT, 8), 0, s>>>(in, out, A, ny, B);
  } else {
    // external [z][y][x] <-> internal [y][z][x]
    const int A = to_internal ? nz : ny, B = to_internal ? ny : nz;
    const long long rows = (long long)A * B;
    k_swap_outer<<<(unsigned)std::min<long long>(rows, 152 * 16), 128, 0, s>>>(in, out, A, B, nx);
  }
  FDI_LAUNCH_CHECK(p);
  return FDI_OK;
}

}  // namespace fdi
