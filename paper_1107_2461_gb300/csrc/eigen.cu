// Plan-time generalised eigen decomposition of the 1D operators (Sec. 3, Eq. 24).
//
// D = M^{-1} K with M diagonal and K symmetric tridiagonal, so
//   S = M^{-1/2} K M^{-1/2} = Q Lambda Q^T,   E = M^{-1/2} Q,   E^{-1} = Q^T M^{1/2} = E^T M.
// S is symmetric tridiagonal; its eigenpairs are found by the implicit QL
// algorithm with Wilkinson-type shifts (Bowdler, Martin, Reinsch & Wilkinson,
// Numer. Math. 11, 1968), in FP64.  One CTA per operator: thread 0 chases the
// bulge along the tridiagonal and records each plane rotation, then all threads
// apply the recorded rotations to their rows of the eigenvector matrix.  The
// paper computes these decompositions once per grid in O(n^3) and neglects
// their cost (Sec. 3).
//
// For a zero-flux operator the null pair is set exactly: Lambda = 0 with the
// constant eigenvector (the reading of Eq. 28 used throughout).
#include <cmath>
#include <mutex>
#include <string>

#include "fdi_internal.h"

namespace fdi {
namespace {

struct EigenJob {
  int n;
  int zero_flux;
  const double* m;
  const double* kd;
  const double* ko;
  double* lam;
  double* E;
  double* Einv;  // also the Z^T scratch during the iteration
};

constexpr int kEigThreads = 256;
constexpr int kMaxQLIter = 60;

__global__ void __launch_bounds__(kEigThreads) k_eigen(const EigenJob* jobs, int* err) {
  const EigenJob job = jobs[blockIdx.x];
  const int n = job.n;
  const int tid = threadIdx.x;
  __shared__ double d[kMaxN], e[kMaxN], rc[kMaxN], rs[kMaxN], sq[kMaxN];
  __shared__ int perm[kMaxN];
  __shared__ int sh_m, sh_iend, sh_state;
  double* Zt = job.Einv;  // Zt[i*n + r] = Z[r][i]

  for (int i = tid; i < n; i += blockDim.x) sq[i] = sqrt(job.m[i]);
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) {
    d[i] = job.kd[i] / job.m[i];
    e[i] = (i + 1 < n) ? job.ko[i] / (sq[i] * sq[i + 1]) : 0.0;
  }
  for (int idx = tid; idx < n * n; idx += blockDim.x) Zt[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
  __syncthreads();

  const double eps = 2.220446049250313e-16;
  for (int l = 0; l < n; ++l) {
    for (int iter = 0;; ++iter) {
      if (tid == 0) {
        int m;
        for (m = l; m < n - 1; ++m) {
          double dd = fabs(d[m]) + fabs(d[m + 1]);
          if (fabs(e[m]) <= eps * dd) break;
        }
        if (m == l) {
          sh_state = 1;
        } else if (iter >= kMaxQLIter) {
          sh_state = 2;
        } else {
          // shift from the leading 2x2 block, then chase from the bottom up
          double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
          double r = hypot(g, 1.0);
          g = d[m] - d[l] + e[l] / (g + copysign(r, g));
          double s = 1.0, c = 1.0, p = 0.0;
          int i;
          bool underflow = false;
          for (i = m - 1; i >= l; --i) {
            double f = s * e[i], b = c * e[i];
            r = hypot(f, g);
            e[i + 1] = r;
            if (r == 0.0) {
              d[i + 1] -= p;
              e[m] = 0.0;
              underflow = true;
              break;
            }
            s = f / r;
            c = g / r;
            g = d[i + 1] - p;
            r = (d[i] - g) * s + 2.0 * c * b;
            p = s * r;
            d[i + 1] = g + p;
            g = c * r - b;
            rc[i] = c;
            rs[i] = s;
          }
          if (!underflow) {
            d[l] -= p;
            e[l] = g;
            e[m] = 0.0;
          }
          sh_m = m;
          sh_iend = underflow ? i + 1 : l;
          sh_state = 0;
        }
      }
      __syncthreads();
      const int state = sh_state;
      if (state != 0) {
        if (state == 2 && tid == 0) atomicExch(err, 1);
        break;
      }
      const int mm = sh_m, iend = sh_iend;
      for (int r = tid; r < n; r += blockDim.x) {
        for (int i = mm - 1; i >= iend; --i) {
          double c = rc[i], s = rs[i];
          double zi = Zt[(size_t)i * n + r], zi1 = Zt[(size_t)(i + 1) * n + r];
          Zt[(size_t)(i + 1) * n + r] = s * zi + c * zi1;
          Zt[(size_t)i * n + r] = c * zi - s * zi1;
        }
      }
      __syncthreads();
    }
    __syncthreads();
  }

  // order: descending eigenvalues (the smoothest mode first)
  for (int k = tid; k < n; k += blockDim.x) {
    int rank = 0;
    for (int j = 0; j < n; ++j) rank += (d[j] > d[k]) || (d[j] == d[k] && j < k);
    perm[rank] = k;
  }
  __syncthreads();
  __shared__ double null_norm, null_sign;
  if (tid == 0) {
    double s2 = 0.0, dot = 0.0;
    for (int r = 0; r < n; ++r) {
      s2 += job.m[r];
      dot += sq[r] * Zt[(size_t)perm[0] * n + r];
    }
    null_norm = sqrt(s2);
    null_sign = dot < 0.0 ? -1.0 : 1.0;
  }
  __syncthreads();
  if (job.zero_flux) {
    // the other eigenvectors are orthogonal to the exact null vector: project
    // out the component the rounding left along it and renormalise
    for (int k = 1 + tid; k < n; k += blockDim.x) {
      double* z = Zt + (size_t)perm[k] * n;
      double dot = 0.0;
      for (int r = 0; r < n; ++r) dot += sq[r] * z[r];
      dot /= null_norm;
      double nrm = 0.0;
      for (int r = 0; r < n; ++r) {
        z[r] -= dot * sq[r] / null_norm;
        nrm += z[r] * z[r];
      }
      const double inv = 1.0 / sqrt(nrm);
      for (int r = 0; r < n; ++r) z[r] *= inv;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    int r = idx / n, k = idx % n;
    double q = Zt[(size_t)perm[k] * n + r];
    if (job.zero_flux && k == 0) q = null_sign * sq[r] / null_norm;
    job.E[idx] = q / sq[r];
  }
  for (int k = tid; k < n; k += blockDim.x)
    job.lam[k] = (job.zero_flux && k == 0) ? 0.0 : d[perm[k]];
  __syncthreads();
  // E^{-1} = E^T M  (row k of E^{-1} = column k of E scaled by the widths)
  for (int idx = tid; idx < n * n; idx += blockDim.x) {
    int k = idx / n, r = idx % n;
    job.Einv[idx] = job.E[(size_t)r * n + k] * job.m[r];
  }
}

}  // namespace

namespace {
fdi_status run_jobs(const std::vector<EigenJob>& jobs, cudaStream_t s, int* d_err);
}

fdi_status eigen_decompose_all(const std::vector<Axis*>& axes, cudaStream_t s, int* d_err) {
  std::vector<EigenJob> jobs;
  for (Axis* ax : axes)
    if (!ax->periodic)
      jobs.push_back(EigenJob{ax->n, ax->zero_flux ? 1 : 0, ax->m, ax->kd, ax->ko, ax->lam, ax->E, ax->Einv});
  return run_jobs(jobs, s, d_err);
}

fdi_status eigen_decompose_batch(int count, int n, const double* m, const double* kd_all, const double* ko,
                                 bool zero_flux0, double* lam_all, double* E_all, double* Einv_all, cudaStream_t s,
                                 int* d_err) {
  std::vector<EigenJob> jobs;
  for (int q = 0; q < count; ++q)
    jobs.push_back(EigenJob{n, (q == 0 && zero_flux0) ? 1 : 0, m, kd_all + (size_t)q * n, ko,
                            lam_all + (size_t)q * n, E_all + (size_t)q * n * n, Einv_all + (size_t)q * n * n});
  return run_jobs(jobs, s, d_err);
}

namespace {
fdi_status run_jobs(const std::vector<EigenJob>& jobs, cudaStream_t s, int* d_err) {
  if (jobs.empty()) return FDI_OK;
  EigenJob* d_jobs = nullptr;
  FDI_CUDA_TRY(cudaMalloc(&d_jobs, jobs.size() * sizeof(EigenJob)));
  cudaError_t e = cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(EigenJob),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    k_eigen<<<(unsigned)jobs.size(), kEigThreads, 0, s>>>(d_jobs, d_err);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_jobs);
  if (e != cudaSuccess) {
    set_error(std::string("eigen decomposition: ") + cudaGetErrorString(e));
    return FDI_ERR_CUDA;
  }
  return FDI_OK;
}
}  // namespace

// ---------------------------------------------------------------------------
// Allocation-free variant of the eigen decomposition.
//
// For callers that may not allocate device memory (code running where
// cudaMalloc is forbidden or unsafe, such as allocation-free real-time loops or
// runtimes that own every device allocation) and that still want the 1D
// eigenbasis of a new grid: the kernel's scratch -- the 1D operator it reads,
// its job descriptor and its convergence flag -- lives in the file-scope array
// below instead of in buffers allocated per call.  The eigenvector matrix is
// accumulated in the caller's E^{-1} output, as in the plan path.
namespace {

constexpr int kNoallocMaxDevices = 64;
// layout: m[kMaxN] | kd[kMaxN] | ko[kMaxN] | job (8 doubles) | flag (8 doubles)
constexpr int kNoallocDoubles = 3 * kMaxN + 16;
static __device__ __align__(256) double g_eigen_scratch[kNoallocDoubles];
static double* g_eigen_scratch_ptr[kNoallocMaxDevices] = {};
static std::mutex g_eigen_scratch_mu;

static_assert(sizeof(EigenJob) <= 8 * sizeof(double), "job slot too small");

}  // namespace
}  // namespace fdi

extern "C" fdi_status fdi_eigen_noalloc(const double* faces, int n, int face_kind, fdi_bc bc_lo, fdi_bc bc_hi,
                                        double* lam, double* E, double* Einv, int* converged,
                                        fdi_stream_t stream) {
  using namespace fdi;
  if (!faces || !lam || !E || !Einv) return FDI_ERR_INVALID_ARG;
  if (face_kind != 0 && face_kind != 1) return FDI_ERR_INVALID_ARG;
  if ((unsigned)bc_lo > 1u || (unsigned)bc_hi > 1u) return FDI_ERR_INVALID_ARG;
  if (face_kind == 1 && (bc_lo != FDI_BC_DIRICHLET || bc_hi != FDI_BC_DIRICHLET)) {
    set_error("fdi_eigen_noalloc: a face operator (face_kind 1) has no-slip walls; bc_lo and bc_hi must be "
              "FDI_BC_DIRICHLET");
    return FDI_ERR_INVALID_ARG;
  }
  if (n < (face_kind ? 3 : 2) || n > kMaxN) {
    set_error("fdi_eigen_noalloc: n must lie in [2, 256] (cell) or [3, 256] (face); its scratch holds 256 unknowns");
    return FDI_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n; ++i)
    if (!(faces[i + 1] > faces[i]) || !std::isfinite(faces[i]) || !std::isfinite(faces[i + 1])) {
      set_error("fdi_eigen_noalloc: faces must be finite and strictly ascending");
      return FDI_ERR_INVALID_ARG;
    }
  // 1D finite-volume operator on the stack (no heap allocation)
  double m[kMaxN], kd[kMaxN], ko[kMaxN];
  int u = n;
  bool zero_flux = false;
  if (face_kind == 0) {
    for (int i = 0; i < n; ++i) {
      m[i] = faces[i + 1] - faces[i];
      kd[i] = 0.0;
      ko[i] = 0.0;
    }
    for (int i = 0; i + 1 < n; ++i) {
      const double g = 1.0 / (0.5 * (faces[i + 1] + faces[i + 2]) - 0.5 * (faces[i] + faces[i + 1]));
      ko[i] = g;
      kd[i] -= g;
      kd[i + 1] -= g;
    }
    if (bc_lo == FDI_BC_DIRICHLET) kd[0] -= 2.0 / m[0];
    if (bc_hi == FDI_BC_DIRICHLET) kd[n - 1] -= 2.0 / m[n - 1];
    zero_flux = bc_lo == FDI_BC_NEUMANN && bc_hi == FDI_BC_NEUMANN;
  } else {
    u = n - 1;
    for (int j = 1; j < n; ++j) {
      m[j - 1] = 0.5 * (faces[j] + faces[j + 1]) - 0.5 * (faces[j - 1] + faces[j]);
      kd[j - 1] = 0.0;
      ko[j - 1] = 0.0;
    }
    for (int i = 0; i < n; ++i) {
      const double g = 1.0 / (faces[i + 1] - faces[i]);
      const int a = i - 1, b = i;
      if (a >= 0 && a < u) kd[a] -= g;
      if (b >= 0 && b < u) kd[b] -= g;
      if (a >= 0 && b < u) ko[a] = g;
    }
  }
  // per-device set-up: the device address of the scratch array
  int dev = 0;
  FDI_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return FDI_ERR_UNSUPPORTED;
  double* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_eigen_scratch_mu);
    if (!g_eigen_scratch_ptr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_eigen_scratch);
      if (e != cudaSuccess || !ptr) {
        set_error(std::string("fdi_eigen_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return FDI_ERR_CUDA;
      }
      g_eigen_scratch_ptr[dev] = static_cast<double*>(ptr);
    }
    base = g_eigen_scratch_ptr[dev];
  }
  double* d_m = base;
  double* d_kd = base + kMaxN;
  double* d_ko = base + 2 * kMaxN;
  EigenJob* d_job = reinterpret_cast<EigenJob*>(base + 3 * kMaxN);
  int* d_flag = reinterpret_cast<int*>(base + 3 * kMaxN + 8);
  const EigenJob job{u, zero_flux ? 1 : 0, d_m, d_kd, d_ko, lam, E, Einv};
  cudaStream_t s = (cudaStream_t)stream;
  // the operator is copied from pageable host memory (the stack), which a
  // stream capture cannot record: refuse instead of breaking the capture
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    set_error("fdi_eigen_noalloc: the stream is being captured; this call copies from pageable host memory and "
              "must run outside stream capture");
    return FDI_ERR_INVALID_ARG;
  }
  // pageable-source copies return once the source has been staged, so the
  // stack arrays may go out of scope afterwards
  FDI_CUDA_TRY(cudaMemcpyAsync(d_m, m, u * sizeof(double), cudaMemcpyHostToDevice, s));
  FDI_CUDA_TRY(cudaMemcpyAsync(d_kd, kd, u * sizeof(double), cudaMemcpyHostToDevice, s));
  FDI_CUDA_TRY(cudaMemcpyAsync(d_ko, ko, u * sizeof(double), cudaMemcpyHostToDevice, s));
  FDI_CUDA_TRY(cudaMemcpyAsync(d_job, &job, sizeof(EigenJob), cudaMemcpyHostToDevice, s));
  FDI_CUDA_TRY(cudaMemsetAsync(d_flag, 0, sizeof(int), s));  // the flag keeps the last call's value
  k_eigen<<<1, kEigThreads, 0, s>>>(d_job, d_flag);
  FDI_CUDA_TRY(cudaGetLastError());
  if (converged) {
    int flag = 0;
    FDI_CUDA_TRY(cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    FDI_CUDA_TRY(cudaStreamSynchronize(s));
    *converged = flag == 0 ? 1 : 0;
  }
  return FDI_OK;
}
