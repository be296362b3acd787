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

fdi_status eigen_decompose_all(const std::vector<Axis*>& axes, cudaStream_t s, int* d_err) {
  std::vector<EigenJob> jobs;
  for (Axis* ax : axes)
    jobs.push_back(EigenJob{ax->n, ax->zero_flux ? 1 : 0, ax->m, ax->kd, ax->ko, ax->lam, ax->E, ax->Einv});
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

}  // namespace fdi
