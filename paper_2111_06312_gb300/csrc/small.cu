// Small l x l FP64 step of CholeskyQR (Alg. 2, right), one CTA (l <= 160):
// Cholesky of the Gram matrix Q^T Q with an adaptive diagonal shift and the
// inverse of the triangular factor.  (The Rayleigh-Ritz SVD is in jacobi.cu.)
#include <mutex>

#include "internal.h"

namespace isvd {
namespace {

constexpr int kSmallThreads = 1024;

__device__ __forceinline__ bool pass_skipped(const int32_t *state, int32_t pass) {
  return pass > 2 && state[0] + 2 < pass;
}

// Cholesky W = R^T R (R upper) in shared memory, then R^-1 in place.
// A pivot that is not positive and finite triggers a retry with W + shift I,
// shift = 16 l u tr(W) (u = unit roundoff of the stored block) growing
// tenfold per retry (shifted CholeskyQR, Fukaya et al. 2020, with a shift
// sized to the rounding of an FP32-accumulated Gram).  A shifted pass records
// itself in state[0] so that two plain passes follow it.
__global__ void __launch_bounds__(kSmallThreads) chol_inv_kernel(const double *__restrict__ W, int32_t l,
                                                                 double unit_roundoff, float *__restrict__ Rinv,
                                                                 int64_t ldr, double *__restrict__ Rout,
                                                                 double *__restrict__ Racc,
                                                                 double *__restrict__ tmp, int32_t *state,
                                                                 isvd_info *info, int32_t pass) {
  if (pass_skipped(state, pass)) return;
  extern __shared__ double A[];  // l * l, then l for a column buffer
  double *col = A + (size_t)l * l;
  __shared__ int fail;
  __shared__ double trace;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0 && state[2]) atomicExch(&info->status, (int)ISVD_ERR_TIMEOUT);  // a Gram wait gave up
  if (tid == 0) {
    double t = 0.0;
    for (int i = 0; i < l; ++i) t += W[(size_t)i * l + i];
    trace = t;
  }
  __syncthreads();
  double shift = 0.0;
  int ok = 0;
  for (int attempt = 0; attempt < 10 && !ok; ++attempt) {
    if (attempt == 1) shift = 16.0 * l * unit_roundoff * fabs(trace);
    if (attempt > 1) shift *= 10.0;
    for (int idx = tid; idx < l * l; idx += nt) {
      const int i = idx / l, c = idx - i * l;
      A[idx] = W[idx] + (i == c ? shift : 0.0);
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < l; ++j) {
      if (tid == 0) {
        const double d = A[(size_t)j * l + j];
        if (!(d > 0.0) || !isfinite(d)) fail = 1;
        else A[(size_t)j * l + j] = sqrt(d);
      }
      __syncthreads();
      if (fail) break;
      const double rjj = A[(size_t)j * l + j];
      for (int c = j + 1 + tid; c < l; c += nt) A[(size_t)j * l + c] /= rjj;
      __syncthreads();
      const int m = l - j - 1;
      for (int idx = tid; idx < m * m; idx += nt) {
        const int ii = idx / m, cc = idx - ii * m;
        if (cc >= ii) {
          const int i = j + 1 + ii, c = j + 1 + cc;
          A[(size_t)i * l + c] -= A[(size_t)j * l + i] * A[(size_t)j * l + c];
        }
      }
      __syncthreads();
    }
    ok = !fail;
    __syncthreads();
  }
  if (!ok) {
    // breakdown even with shifts (non-finite input): identity, flag the error
    if (tid == 0) {
      state[1] = 1;
      atomicExch(&info->status, (int)ISVD_ERR_NOT_POSITIVE_DEFINITE);
    }
    for (int idx = tid; idx < l * l; idx += nt) {
      const int i = idx / l, c = idx - i * l;
      A[idx] = (i == c) ? 1.0 : 0.0;
    }
    __syncthreads();
  } else if (tid == 0) {
    if (shift > 0.0) {
      atomicMax(&state[0], pass);
      atomicAdd(&info->chol_shifts, 1);
    }
    atomicAdd(&info->cholqr_passes, 1);
  }
  // from pass 2 on, a factor far from I schedules one more pass (see chol_cluster.cu)
  if (ok && pass >= 2) {
    __shared__ int far_from_identity;
    if (tid == 0) far_from_identity = 0;
    __syncthreads();
    for (int idx = tid; idx < l * l; idx += nt) {
      const int i = idx / l, c = idx - i * l;
      if (c >= i && fabs(A[idx] - (i == c ? 1.0 : 0.0)) > 0.25) far_from_identity = 1;
    }
    __syncthreads();
    if (tid == 0 && far_from_identity) atomicMax(&state[0], pass - 1);
  }
  // zero the strict lower triangle
  for (int idx = tid; idx < l * l; idx += nt) {
    const int i = idx / l, c = idx - i * l;
    if (c < i) A[idx] = 0.0;
  }
  __syncthreads();
  if (Rout)
    for (int idx = tid; idx < l * l; idx += nt) Rout[idx] = A[idx];
  if (Racc) {
    // Racc <- R Racc (both upper triangular)
    for (int idx = tid; idx < l * l; idx += nt) {
      const int i = idx / l, c = idx - i * l;
      double s = 0.0;
      for (int t = i; t <= c; ++t) s += A[(size_t)i * l + t] * Racc[(size_t)t * l + c];
      tmp[idx] = (c >= i) ? s : 0.0;
    }
    __syncthreads();
    for (int idx = tid; idx < l * l; idx += nt) Racc[idx] = tmp[idx];
  }
  __syncthreads();
  // in-place inverse of the upper triangular R, column by column:
  // S_jj = 1/R_jj, S_ij = -(sum_{k=i}^{j-1} S_ik R_kj) / R_jj  (i < j)
  for (int j = 0; j < l; ++j) {
    if (tid < j) {
      double s = 0.0;
      for (int k = tid; k < j; ++k) s += A[(size_t)tid * l + k] * A[(size_t)k * l + j];
      col[tid] = s;
    }
    __syncthreads();
    const double inv = 1.0 / A[(size_t)j * l + j];
    if (tid < j) A[(size_t)tid * l + j] = -col[tid] * inv;
    __syncthreads();
    if (tid == 0) A[(size_t)j * l + j] = inv;
    __syncthreads();
  }
  for (int idx = tid; idx < l * (int)ldr; idx += nt) {
    const int i = idx / (int)ldr, c = idx - i * (int)ldr;
    Rinv[(size_t)i * ldr + c] = (c < l) ? (float)A[(size_t)i * l + c] : 0.f;
  }
}

__global__ void orth_reset_kernel(int32_t *state) {
  if (threadIdx.x < kOrthStateInts) state[threadIdx.x] = 0;
}

__global__ void racc_init_kernel(double *Racc, int32_t l) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < l * l; idx += gridDim.x * blockDim.x)
    Racc[idx] = (idx / l == idx % l) ? 1.0 : 0.0;
}

size_t chol_smem(int32_t l) { return sizeof(double) * ((size_t)l * l + l); }

}  // namespace

cudaError_t small_kernels_init() {
  static cudaError_t err = cudaSuccess;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaError_t e = cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)chol_smem(ISVD_MAX_BLOCK));
    chol_cluster_size();  // attributes and the cluster size of the distributed form
    err = e;
  });
  return err;
}

cudaError_t orth_reset_launch(int32_t *state, cudaStream_t s) {
  orth_reset_kernel<<<1, 32, 0, s>>>(state);
  return cudaGetLastError();
}

cudaError_t racc_init_launch(double *Racc, int32_t l, cudaStream_t s) {
  racc_init_kernel<<<(unsigned)ceil_div((int64_t)l * l, 256), 256, 0, s>>>(Racc, l);
  return cudaGetLastError();
}

cudaError_t chol_inv_launch(const double *W, int32_t l, int64_t rows, int dtype, float *Rinv, int64_t ldr, double *R,
                            double *Racc, double *tmp, int32_t *state, isvd_info *info, int32_t pass,
                            cudaStream_t s) {
  (void)rows;
  (void)dtype;  // the Gram is accumulated in FP32 for both storage types
  const double u = 5.9604644775390625e-08;
  // blocks of at least 32 columns go to the cluster form when the GPU can host it
  if (l >= 32 && chol_cluster_size() >= 8)
    return chol_cluster_launch(W, l, u, Rinv, ldr, R, Racc, tmp, state, info, pass, s);
  chol_inv_kernel<<<1, kSmallThreads, chol_smem(l), s>>>(W, l, u, Rinv, ldr, R, Racc, tmp, state, info, pass);
  return cudaGetLastError();
}

}  // namespace isvd
