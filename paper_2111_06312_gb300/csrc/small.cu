// Small l x l FP64 steps of the randomized SVD, one CTA each (l <= 160):
//  - Cholesky of the Gram matrix Q^T Q with an adaptive diagonal shift and
//    the inverse of the triangular factor (CholeskyQR, Alg. 2, right);
//  - one-sided Jacobi SVD for the Rayleigh-Ritz step of Alg. 1.
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
      state[0] = pass;
      atomicAdd(&info->chol_shifts, 1);
    }
    atomicAdd(&info->cholqr_passes, 1);
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

// One-sided Jacobi on the columns of G = A^T (column p of G is row p of A,
// kept contiguous in shared memory).  Pairs follow the round-robin
// tournament order, l/2 disjoint pairs per round, one warp per pair.
// Rotation: Rutishauser's formula; convergence when every pair satisfies
// |g_p.g_q| <= tol ||g_p|| ||g_q|| with tol = max(1e-15, sqrt(l) eps).
// Then A^T = (G J Sigma^-1) Sigma J^T, i.e. A = J Sigma (G J Sigma^-1)^T:
// Uo = J, Vo = normalised rotated columns, S descending.
__global__ void __launch_bounds__(kSmallThreads) jacobi_kernel(const double *__restrict__ A, int32_t l,
                                                               double *__restrict__ Uo, double *__restrict__ S,
                                                               double *__restrict__ Vo, double *__restrict__ Jt,
                                                               float *__restrict__ Uk, float *__restrict__ Vk,
                                                               float *__restrict__ Sk, int32_t k, isvd_info *info,
                                                               int32_t iters) {
  extern __shared__ double Gs[];  // [l2][l2]
  __shared__ double nrm[ISVD_MAX_BLOCK + 2];
  __shared__ int perm[ISVD_MAX_BLOCK + 2];
  __shared__ double fro2;
  const int l2 = (l + 1) & ~1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
  for (int idx = tid; idx < l2 * l2; idx += nt) {
    const int p = idx / l2, i = idx - p * l2;
    Gs[idx] = (p < l && i < l) ? A[(size_t)p * l + i] : 0.0;
    Jt[idx] = (p == i) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    double f = 0.0;
    for (int idx = 0; idx < l2 * l2; ++idx) f += Gs[idx] * Gs[idx];
    fro2 = f;
  }
  __syncthreads();
  const double eps = 2.220446049250313e-16;
  const double tol = fmax(1e-15, sqrt((double)l2) * eps);
  const double tiny = (double)l2 * eps * (double)l2 * eps * fro2;
  for (int sweep = 0; sweep < 60; ++sweep) {
    int rotated = 0;
    for (int round = 0; round < l2 - 1; ++round) {
      for (int pi = warp; pi < l2 / 2; pi += nwarp) {
        int p, q;
        if (pi == 0) {
          p = round;
          q = l2 - 1;
        } else {
          p = (round + pi) % (l2 - 1);
          q = (round - pi + (l2 - 1)) % (l2 - 1);
        }
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int i = lane; i < l2; i += 32) {
          const double gp = Gs[(size_t)p * l2 + i], gq = Gs[(size_t)q * l2 + i];
          al += gp * gp;
          be += gq * gq;
          ga += gp * gq;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          ga += __shfl_xor_sync(0xffffffffu, ga, o);
        }
        if (ga == 0.0 || fabs(ga) <= tol * sqrt(al * be)) continue;
        if (al <= tiny && be <= tiny) continue;
        rotated = 1;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        for (int i = lane; i < l2; i += 32) {
          const double gp = Gs[(size_t)p * l2 + i], gq = Gs[(size_t)q * l2 + i];
          Gs[(size_t)p * l2 + i] = cs * gp - sn * gq;
          Gs[(size_t)q * l2 + i] = sn * gp + cs * gq;
          const double jp = Jt[(size_t)p * l2 + i], jq = Jt[(size_t)q * l2 + i];
          Jt[(size_t)p * l2 + i] = cs * jp - sn * jq;
          Jt[(size_t)q * l2 + i] = sn * jp + cs * jq;
        }
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) break;
  }
  // column norms and descending order
  for (int p = warp; p < l2; p += nwarp) {
    double s = 0.0;
    for (int i = lane; i < l2; i += 32) s += Gs[(size_t)p * l2 + i] * Gs[(size_t)p * l2 + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) nrm[p] = sqrt(s);
  }
  __syncthreads();
  if (tid == 0) {
    for (int p = 0; p < l2; ++p) perm[p] = p;
    for (int a = 1; a < l2; ++a) {  // stable insertion sort, descending
      const int x = perm[a];
      int b = a - 1;
      while (b >= 0 && nrm[perm[b]] < nrm[x]) {
        perm[b + 1] = perm[b];
        --b;
      }
      perm[b + 1] = x;
    }
    if (info) info->iters_done = iters;
  }
  __syncthreads();
  for (int idx = tid; idx < l * l; idx += nt) {
    const int i = idx / l, c = idx - i * l;
    const int p = perm[c];
    const double sg = nrm[p];
    const double v = sg > 0.0 ? Gs[(size_t)p * l2 + i] / sg : 0.0;
    const double u = Jt[(size_t)p * l2 + i];
    if (Vo) Vo[idx] = v;
    if (Uo) Uo[idx] = u;
    if (c < k) {
      if (Vk) Vk[(size_t)i * k + c] = (float)v;
      if (Uk) Uk[(size_t)i * k + c] = (float)u;
    }
  }
  for (int c = tid; c < l; c += nt) {
    if (S) S[c] = nrm[perm[c]];
    if (Sk && c < k) Sk[c] = (float)nrm[perm[c]];
  }
}

size_t chol_smem(int32_t l) { return sizeof(double) * ((size_t)l * l + l); }
size_t jacobi_smem(int32_t l) {
  const size_t l2 = (size_t)((l + 1) & ~1);
  return sizeof(double) * l2 * l2;
}

}  // namespace

cudaError_t small_kernels_init() {
  static cudaError_t err = cudaSuccess;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaError_t e = cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)chol_smem(ISVD_MAX_BLOCK));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)jacobi_smem(ISVD_MAX_BLOCK));
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
  chol_inv_kernel<<<1, kSmallThreads, chol_smem(l), s>>>(W, l, u, Rinv, ldr, R, Racc, tmp, state, info, pass);
  return cudaGetLastError();
}

cudaError_t small_svd_launch(const double *A, int32_t l, double *Uo, double *S, double *Vo, double *work, float *Uk,
                             float *Vk, float *Sk, int32_t k, isvd_info *info, int32_t iters, cudaStream_t s) {
  jacobi_kernel<<<1, kSmallThreads, jacobi_smem(l), s>>>(A, l, Uo, S, Vo, work, Uk, Vk, Sk, k, info, iters);
  return cudaGetLastError();
}

}  // namespace isvd
