// Split-precision tcgen05 transform pass: declarations shared by the solver.
#pragma once
#include <cuda_runtime.h>

#include "fdi_internal.h"

namespace fdi {

// TC_OUT_F32: out = T x.  TC_OUT_DF_ADD: (out, out_lo) += T x, the two FP32
// planes holding one double-float value per element, renormalised on store
// (row-major outputs only)
enum { TC_OUT_F32 = 0, TC_OUT_DF_ADD = 1 };

// A transform matrix T (n x n, output index k, input index j) prepared for the
// tensor cores: B = [hi; lo] fp16 [2*N_pad][K_pad], per-row power-of-two scale
// undone by col_scale[k], and its TMA descriptor.
struct TcMatrix {
  int n = 0, N_pad = 0, K_pad = 0;
  void* B = nullptr;
  float* col_scale = nullptr;
  // TMA descriptor of B (boxes of N_pad rows x 32 columns)
  alignas(64) unsigned char tmap[128];
};

struct TcArgs {
  // input: rows of K contiguous FP32 values, row r at in + r * in_pitch
  // (K-major); or, with a_mn, the transposed layout: element (r, k) at
  //   in + ((r / a_mslab) * K + k) * in_pitch + r % a_mslab
  // (a_rows rows of in_pitch values, a_mslab % 128 == 0)
  const float* in = nullptr;
  long long R = 0;
  int K = 0;
  int in_pitch = 0;
  int a_mn = 0;
  long long a_mslab = 0, a_rows = 0;
  const float* scale_in = nullptr;  // device: max |in| (sets the fp16 scaling)
  // output: element (r, k) of an FP32 field at
  //   (r / S) * slab_stride + (r % S) * row_stride + k * col_stride
  int mode = TC_OUT_F32;
  int n_out = 0;
  float* out_f32 = nullptr;
  float* out_lo = nullptr;          // TC_OUT_DF_ADD: low plane, same layout as out_f32
  int lo_valid = 1;                 // TC_OUT_DF_ADD: 0 = the low plane holds no value yet (read as 0)
  long long S = 1, slab_stride = 0, row_stride = 0, col_stride = 1;
  float* scale_out = nullptr;       // device: atomic max |out| (next pass's scaling)
  // set by the launcher: 0 thread stores; 1 TMA stores of a transposed output
  // (3D map over (row in slab, column, slab)); 2 TMA stores of a row-major
  // output (2D map over (column, row))
  int tma_store = 0;
  const int* skip = nullptr;
  int* err = nullptr;
  int pdl = 0;                      // launch with programmatic stream serialization
  long long wait_cycles = 0;        // bound of every wait (cycles); 0: the default
  // filled by the launcher
  int N_pad = 0, nK = 0;
  // tiles at and past n_full (the last, partial wave of a multi-wave grid) run
  // as two half-width items of N_pad / 2 output columns each
  long long n_full = 0;
  const float* col_scale = nullptr;
};

fdi_status tc_prepare_matrix(fdi_plan* p, const double* T, int n, TcMatrix* m, cudaStream_t s);
void tc_free_matrix(TcMatrix* m);
// the matrix in the resident solve's shared-memory layout (K chunks of 32:
// hi rows, lo rows, 64-byte swizzle); cudaMalloc'ed, the caller frees it
fdi_status tc_resident_image(fdi_plan* p, const TcMatrix& m, uint8_t** img, cudaStream_t s);
fdi_status launch_tc_transform(fdi_plan* p, const TcMatrix& m, TcArgs args, const char* name, cudaStream_t s);

}  // namespace fdi
