// The l x l FP64 step of CholeskyQR (Alg. 2, right) spread over a
// thread-block cluster: Cholesky W = R^T R with the adaptive shift of
// small.cu, then R^-1 (FP32 copy for the tensor-core product Q R^-1), the
// optional FP64 R and the running product Racc <- R Racc.
//
// GB300 runs FP64 at about 2 FMA per clock per SM, so the ~l^3/3 FMA of the
// factorisation and the ~l^3/6 of the inverse take about a millisecond on one
// SM; here CL CTAs (8 or 16) each own the columns c = rank (mod CL):
//   - factorisation: right-looking, in panels of kNB rows (8: measured
//     faster than 16 and 32 at l = 144).  Every CTA reads
//     the kNB x kNB diagonal block from its owners through distributed shared
//     memory and factors it itself (identical arithmetic, so every CTA takes
//     the same decisions about a failed pivot); each CTA solves the panel
//     rows of its own columns, then reads the whole panel and updates its own
//     columns of the trailing matrix (two cluster barriers per panel);
//   - inverse: every CTA gathers the packed upper triangle of R and computes
//     its own columns of R^-1 by back substitution, one warp per column.
#include <cooperative_groups.h>

#include <mutex>

#include "internal.h"

namespace cg = cooperative_groups;

// preferred cluster size of the Cholesky (16 or 8; 8 when 16 cannot be resident)
#ifndef ISVD_CHOL_CLUSTER
#define ISVD_CHOL_CLUSTER 16
#endif

namespace isvd {
namespace {

constexpr int kCholThreads = 512;
#ifndef ISVD_CHOL_NB
#define ISVD_CHOL_NB 8
#endif
constexpr int kNB = ISVD_CHOL_NB;  // panel rows (at most 32: the panel solve keeps one row per lane)
constexpr double kReorthThreshold = 0.25;

__host__ __device__ inline int cols_per_cta(int l, int cl) { return (l + cl - 1) / cl; }
__host__ __device__ inline size_t packed_size(int l) { return (size_t)l * (l + 1) / 2; }
__device__ __forceinline__ int packed_off(int i, int l) { return i * l - i * (i - 1) / 2; }  // row i starts here

// shared memory (doubles): Acol[cpc][l] | D[kNB][kNB + 1] | invD[kNB] | X (max(kNB * l, packed l)) | invd[l] | xbuf[16][l]
__host__ __device__ inline size_t chol_cluster_smem(int l, int cl) {
  const size_t x = (size_t)kNB * l > packed_size(l) ? (size_t)kNB * l : packed_size(l);
  return sizeof(double) * ((size_t)cols_per_cta(l, cl) * l + kNB * (kNB + 1) + kNB + x + l +
                           (size_t)(kCholThreads / 32) * l);
}

__device__ __forceinline__ bool pass_skipped(const int32_t *state, int32_t pass) {
  return pass > 2 && state[0] + 2 < pass;
}

__global__ void __launch_bounds__(kCholThreads, 1) chol_cluster_kernel(const double *__restrict__ W, int32_t l,
                                                                    double unit_roundoff, float *__restrict__ Rinv,
                                                                    int64_t ldr, double *__restrict__ Rout,
                                                                    double *__restrict__ Racc,
                                                                    double *__restrict__ tmp, int32_t *state,
                                                                    isvd_info *info, int32_t pass) {
  if (pass_skipped(state, pass)) return;  // uniform over the cluster
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
  const int cpc = cols_per_cta(l, CL);
  extern __shared__ double sm[];
  double *Acol = sm;                                   // own column cc (global c = rank + cc CL), rows 0..l-1
  double *D = Acol + (size_t)cpc * l;                  // diagonal block, D[r * (kNB + 1) + c]
  double *invD = D + kNB * (kNB + 1);
  double *X = invD + kNB;                              // panel P[t * l + i] or packed R
  const size_t xsz = (size_t)kNB * l > packed_size(l) ? (size_t)kNB * l : packed_size(l);
  double *invd = X + xsz;
  double *xbuf = invd + l;
  __shared__ int s_fail;
  __shared__ double s_trace;

  if (warp == 0) {
    // trace of W: lanes over the diagonal, then a fixed-order reduction
    double t = 0.0;
    for (int i = lane; i < l; i += 32) t += W[(size_t)i * l + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) {
      s_trace = t;
      if (rank == 0 && state[2]) atomicExch(&info->status, (int)ISVD_ERR_TIMEOUT);  // a Gram wait gave up
    }
  }
  __syncthreads();

  double shift = 0.0;
  bool ok = false;
  for (int attempt = 0; attempt < 10 && !ok; ++attempt) {
    if (attempt == 1) shift = 16.0 * l * unit_roundoff * fabs(s_trace);
    if (attempt > 1) shift *= 10.0;
    if (attempt > 0) cluster.sync();  // nobody still reads the previous attempt's columns
    for (int idx = tid; idx < cpc * l; idx += nt) {
      const int cc = idx / l, i = idx - cc * l;
      const int c = rank + cc * CL;
      Acol[idx] = (c < l && i <= c) ? W[(size_t)i * l + c] + (i == c ? shift : 0.0) : 0.0;
    }
    if (tid == 0) s_fail = 0;
    cluster.sync();
    bool failed = false;
    for (int k0 = 0; k0 < l; k0 += kNB) {
      const int nb = (l - k0) < kNB ? (l - k0) : kNB;
      // (a) diagonal block from the owners of its columns
      for (int idx = tid; idx < nb * nb; idx += nt) {
        const int r = idx / nb, c = idx - r * nb;
        const int gc = k0 + c;
        double v = 0.0;
        if (r <= c) v = cluster.map_shared_rank(Acol, gc % CL)[(size_t)(gc / CL) * l + k0 + r];
        D[r * (kNB + 1) + c] = v;
      }
      __syncthreads();
      // (b) factor it (one warp): row j scaled by 1/sqrt(d_jj), then the
      // trailing triangle updated with one lane per element
      if (warp == 0) {
        for (int j = 0; j < nb; ++j) {
          const double d = D[j * (kNB + 1) + j];
          if (!(d > 0.0) || !isfinite(d)) {
            if (lane == 0) s_fail = 1;
            break;
          }
          const double inv = rsqrt(d);
          __syncwarp();
          if (lane == j) {
            D[j * (kNB + 1) + j] = d * inv;
            invD[j] = inv;
          }
          if (lane > j && lane < nb) D[j * (kNB + 1) + lane] *= inv;
          __syncwarp();
          const int m = nb - j - 1;  // trailing order
          for (int idx = lane; idx < m * m; idx += 32) {
            const int ii = idx / m, cc = idx - ii * m;
            if (cc >= ii) {
              const int i = j + 1 + ii, c = j + 1 + cc;
              D[i * (kNB + 1) + c] -= D[j * (kNB + 1) + i] * D[j * (kNB + 1) + c];
            }
          }
          __syncwarp();
        }
      }
      __syncthreads();
      if (s_fail) {
        failed = true;
        break;  // every CTA factors the same block, so all leave here together
      }
      // (c) panel rows k0..k0+nb of the own columns, one warp per column
      for (int cc = warp; cc < cpc; cc += nt / 32) {
        const int c = rank + cc * CL;
        if (c < k0 || c >= l) continue;
        double *a = Acol + (size_t)cc * l + k0;
        if (c < k0 + nb) {
          if (lane <= c - k0) a[lane] = D[lane * (kNB + 1) + (c - k0)];
        } else {
          // solve D^T x = a (D upper), lane r holding row r: once x_r is
          // final (x_r = a_r / D_rr), every later row s subtracts D_rs x_r
          double x = lane < nb ? a[lane] : 0.0;
          for (int r = 0; r < nb; ++r) {
            const double xr = __shfl_sync(0xffffffffu, x, r) * invD[r];
            if (lane == r) x = xr;
            else if (lane > r && lane < nb) x = fma(-D[r * (kNB + 1) + lane], xr, x);
          }
          if (lane < nb) a[lane] = x;
        }
      }
      cluster.sync();
      const int k1 = k0 + nb;
      if (k1 < l) {
        // (e) the whole panel P[t][i] = R[k0 + t][i], i >= k1
        for (int idx = tid; idx < nb * (l - k1); idx += nt) {
          const int t = idx / (l - k1), i = k1 + (idx - t * (l - k1));
          X[(size_t)t * l + i] = cluster.map_shared_rank(Acol, i % CL)[(size_t)(i / CL) * l + k0 + t];
        }
        __syncthreads();
        // (f) trailing update of the own columns
        for (int idx = tid; idx < cpc * l; idx += nt) {
          const int cc = idx / l, i = idx - cc * l;
          const int c = rank + cc * CL;
          if (c < k1 || c >= l || i < k1 || i > c) continue;
          double s = 0.0;
          for (int t = 0; t < nb; ++t) s += X[(size_t)t * l + i] * X[(size_t)t * l + c];
          Acol[idx] -= s;
        }
      }
      cluster.sync();
    }
    ok = !failed;
  }

  // R (or the identity after a breakdown that no shift cured): packed upper triangle in X
  if (ok) {
    for (int idx = tid; idx < l * l; idx += nt) {
      const int c = idx / l, i = idx - c * l;
      if (i <= c) X[packed_off(i, l) + (c - i)] = cluster.map_shared_rank(Acol, c % CL)[(size_t)(c / CL) * l + i];
    }
  } else {
    for (int idx = tid; idx < l * l; idx += nt) {
      const int c = idx / l, i = idx - c * l;
      if (i <= c) X[packed_off(i, l) + (c - i)] = (i == c) ? 1.0 : 0.0;
    }
  }
  cluster.sync();  // no distributed-shared-memory access after this point
  // From pass 2 on, R = chol(Q^T Q) of an already orthonormalised block should
  // be close to I; a factor far from it (max |R - I| > kReorthThreshold) means
  // the block entering this pass was still ill-conditioned, so one more pass
  // is scheduled (the same gate as after a shift).
  if (rank == 0 && ok && pass >= 2) {
    double dev = 0.0;
    for (int idx = tid; idx < l * l; idx += nt) {
      const int i = idx / l, c = idx - i * l;
      if (c >= i) dev = fmax(dev, fabs(X[packed_off(i, l) + (c - i)] - (i == c ? 1.0 : 0.0)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    if (lane == 0 && dev > kReorthThreshold) atomicMax(&state[0], pass - 1);
  }
  if (rank == 0 && tid == 0) {
    if (!ok) {
      state[1] = 1;
      atomicExch(&info->status, (int)ISVD_ERR_NOT_POSITIVE_DEFINITE);
    } else {
      if (shift > 0.0) {
        atomicMax(&state[0], pass);
        atomicAdd(&info->chol_shifts, 1);
      }
      atomicAdd(&info->cholqr_passes, 1);
    }
  }
  for (int i = tid; i < l; i += nt) invd[i] = 1.0 / X[packed_off(i, l)];
  __syncthreads();

  if (Rout)
    for (int idx = tid; idx < cpc * l; idx += nt) {
      const int cc = idx / l, i = idx - cc * l;
      const int c = rank + cc * CL;
      if (c < l) Rout[(size_t)i * l + c] = (i <= c) ? X[packed_off(i, l) + (c - i)] : 0.0;
    }
  if (Racc) {
    // Racc <- R Racc (both upper triangular), own columns, through tmp
    for (int idx = tid; idx < cpc * l; idx += nt) {
      const int cc = idx / l, i = idx - cc * l;
      const int c = rank + cc * CL;
      if (c >= l) continue;
      double s = 0.0;
      for (int t = i; t <= c; ++t) s += X[packed_off(i, l) + (t - i)] * Racc[(size_t)t * l + c];
      tmp[(size_t)i * l + c] = (i <= c) ? s : 0.0;
    }
    cluster.sync();  // every CTA has read Racc
    for (int idx = tid; idx < cpc * l; idx += nt) {
      const int cc = idx / l, i = idx - cc * l;
      const int c = rank + cc * CL;
      if (c < l) Racc[(size_t)i * l + c] = tmp[(size_t)i * l + c];
    }
  }

  // own columns of S = R^-1: S_cc = 1/R_cc, S_ic = -(sum_{t=i+1}^{c} R_it S_tc) / R_ii,
  // one warp per column, right-looking: once S_tc is final (t descending),
  // every row i < t adds R_it S_tc to its running sum x[i] (lanes over i)
  double *x = xbuf + (size_t)warp * l;
  for (int cc = warp; cc < cpc; cc += nt / 32) {
    const int c = rank + cc * CL;
    if (c >= l) break;
    for (int i = lane; i < c; i += 32) x[i] = 0.0;
    __syncwarp();
    for (int t = c; t >= 0; --t) {
      const double xt = t == c ? invd[c] : -x[t] * invd[t];
      for (int i = lane; i < t; i += 32) x[i] = fma(X[packed_off(i, l) + (t - i)], xt, x[i]);
      __syncwarp();
      if (lane == 0) x[t] = xt;
      __syncwarp();
    }
    for (int i = lane; i < l; i += 32) Rinv[(size_t)i * ldr + c] = (i <= c) ? (float)x[i] : 0.f;
    __syncwarp();
  }
  // padding columns l..ldr-1
  for (int c = l + rank; c < ldr; c += CL)
    for (int i = tid; i < l; i += nt) Rinv[(size_t)i * ldr + c] = 0.f;
}

std::once_flag g_once;
cudaError_t g_err = cudaSuccess;
int g_cluster = 1;

}  // namespace

// Largest cluster (16, then 8) that can be resident with the shared memory of
// the largest block; 1 when neither can (the caller then uses one CTA).
int chol_cluster_size() {
  std::call_once(g_once, [] {
    cudaError_t e = cudaFuncSetAttribute(chol_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) cudaGetLastError();
    g_cluster = 1;
    for (int cl : {ISVD_CHOL_CLUSTER, 8}) {
      const size_t smem = chol_cluster_smem(ISVD_MAX_BLOCK, cl);
      if (smem > 227 * 1024) continue;
      e = cudaFuncSetAttribute(chol_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(cl);
      cfg.blockDim = dim3(kCholThreads);
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cl;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, chol_cluster_kernel, &cfg) == cudaSuccess && nclusters > 0) {
        g_cluster = cl;
        break;
      }
      cudaGetLastError();
    }
    g_err = cudaSuccess;
  });
  return g_cluster;
}

cudaError_t chol_cluster_launch(const double *W, int32_t l, double u, float *Rinv, int64_t ldr, double *R,
                                double *Racc, double *tmp, int32_t *state, isvd_info *info, int32_t pass,
                                cudaStream_t s) {
  const int cl = chol_cluster_size();
  if (cl < 8) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(kCholThreads);
  cfg.dynamicSmemBytes = chol_cluster_smem(l, cl);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, chol_cluster_kernel, W, l, u, Rinv, ldr, R, Racc, tmp, state, info, pass);
}

}  // namespace isvd
