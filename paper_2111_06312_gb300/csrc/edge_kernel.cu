// Gaussian-kernel edge function of Sec. 5.1 (App. A.4):
//     f(i, j) = U_i^T E_x[S^x] V_j,  x ~ N(mu, s) truncated to [0.5, 2],
// with the expectation taken on the 301-point grid 0.5, 0.505, ..., 2.0 as
// softmax_x(-(x - mu)^2 exp(s_bar)) (s_bar = log(1 / (2 s^2))), and the link-
// prediction loss of Eq. 9 with its gradient in (mu, s_bar).
//
// The k weights w_c = sum_x pi_x S_c^x and their two derivatives come from one
// CTA in FP64 (k x 301 powers).  Scores and the loss take one warp per pair:
// lane t multiplies columns t, t + 32, ... in FP32, the lane sums are added in
// FP64 by a butterfly, the per-pair loss terms are summed per warp, per CTA
// (warp order) and across a fixed grid of CTAs (CTA order): bitwise
// repeatable.
#include <algorithm>
#include <cmath>

#include "internal.h"

namespace isvd {
namespace {

constexpr int kGrid = 301;                // points of the discretised interval
constexpr double kLo = 0.5, kHi = 2.0;    // the truncation interval
constexpr int kLossBlocks = 2 * kNumSMs;  // fixed grid of the loss kernel

__device__ __forceinline__ double grid_x(int t) { return kLo + (kHi - kLo) * (double)t / (double)(kGrid - 1); }

// w3 = [w | dw/dmu | dw/ds_bar] (FP64, 3k) and, if w3f is not null, the same in FP32.
__global__ void __launch_bounds__(256) edge_weights_kernel(const float *__restrict__ S, int32_t k, double mu,
                                                           double s_bar, double *__restrict__ w3,
                                                           float *__restrict__ w3f) {
  __shared__ double pi[kGrid], dmu[kGrid], ds[kGrid];
  const double e = exp(s_bar);
  if (threadIdx.x == 0) {
    // softmax over the grid of z_x = -(x - mu)^2 e, in a fixed order
    double zmax = -INFINITY;
    for (int t = 0; t < kGrid; ++t) {
      const double d = grid_x(t) - mu;
      ds[t] = -d * d * e;  // z_x (dz/ds_bar = z)
      dmu[t] = 2.0 * d * e;  // dz/dmu
      zmax = fmax(zmax, ds[t]);
    }
    double sum = 0.0;
    for (int t = 0; t < kGrid; ++t) {
      pi[t] = exp(ds[t] - zmax);
      sum += pi[t];
    }
    double mm = 0.0, ms = 0.0;
    for (int t = 0; t < kGrid; ++t) {
      pi[t] /= sum;
      mm += pi[t] * dmu[t];
      ms += pi[t] * ds[t];
    }
    // d pi_x / d theta = pi_x (dz_x/dtheta - sum_y pi_y dz_y/dtheta)
    for (int t = 0; t < kGrid; ++t) {
      dmu[t] = pi[t] * (dmu[t] - mm);
      ds[t] = pi[t] * (ds[t] - ms);
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const double sc = (double)S[c];
    double a = 0.0, b = 0.0, d = 0.0;
    for (int t = 0; t < kGrid; ++t) {
      const double p = sc == 0.0 ? 0.0 : pow(sc, grid_x(t));
      a += pi[t] * p;
      b += dmu[t] * p;
      d += ds[t] * p;
    }
    w3[c] = a;
    w3[k + c] = b;
    w3[2 * k + c] = d;
    if (w3f) {
      w3f[c] = (float)a;
      w3f[k + c] = (float)b;
      w3f[2 * k + c] = (float)d;
    }
  }
}

__device__ __forceinline__ double warp_sum(double t) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  return t;
}

__device__ __forceinline__ float nan_f() { return __int_as_float(0x7fc00000); }

// out[p] = U_src^T diag(w) V_dst, one warp per pair
__global__ void __launch_bounds__(256) edge_scores_kernel(const float *__restrict__ U, int64_t ldu, int64_t rows,
                                                          const float *__restrict__ V, int64_t ldv, int64_t cols,
                                                          int32_t k, const float *__restrict__ w,
                                                          const int32_t *__restrict__ src,
                                                          const int32_t *__restrict__ dst, int64_t n_pairs,
                                                          float *__restrict__ out, isvd_info *info) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < n_pairs; p += nwarp) {
    const int64_t i = __ldg(src + p), j = __ldg(dst + p);
    if (i < 0 || i >= rows || j < 0 || j >= cols) {
      if (lane == 0) {
        out[p] = nan_f();
        if (info) atomicCAS(&info->status, 0, (int)ISVD_ERR_INVALID_ARGUMENT);
      }
      continue;
    }
    const float *ui = U + i * ldu;
    const float *vj = V + j * ldv;
    float f = 0.f;
    for (int c = lane; c < k; c += 32) f = fmaf(__ldg(ui + c) * __ldg(vj + c), __ldg(w + c), f);
    const double t = warp_sum((double)f);
    if (lane == 0) out[p] = (float)t;
  }
}

// Partial sums (per CTA) of the Eq. 9 loss and its gradient in (mu, s_bar):
// pairs 0..n_pos-1 are edges, the next n_neg are non-edges.
__global__ void __launch_bounds__(256) edge_loss_kernel(const float *__restrict__ U, int64_t ldu, int64_t rows,
                                                        const float *__restrict__ V, int64_t ldv, int64_t cols,
                                                        int32_t k, const float *__restrict__ w3,
                                                        const int32_t *__restrict__ pos_src,
                                                        const int32_t *__restrict__ pos_dst, int64_t n_pos,
                                                        const int32_t *__restrict__ neg_src,
                                                        const int32_t *__restrict__ neg_dst, int64_t n_neg,
                                                        double k_neg, double *__restrict__ partial, isvd_info *info) {
  __shared__ double red[8][3];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nwarp = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t total = n_pos + n_neg;
  const double pos_scale = n_pos > 0 ? 1.0 / (double)n_pos : 0.0;
  const double neg_scale = n_neg > 0 ? k_neg / (double)n_neg : 0.0;
  double acc[3] = {0.0, 0.0, 0.0};  // lane 0's running sums
  for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp; p < total; p += nwarp) {
    const bool edge = p < n_pos;
    const int64_t q = edge ? p : p - n_pos;
    const int64_t i = edge ? __ldg(pos_src + q) : __ldg(neg_src + q);
    const int64_t j = edge ? __ldg(pos_dst + q) : __ldg(neg_dst + q);
    if (i < 0 || i >= rows || j < 0 || j >= cols) {
      if (lane == 0) {
        acc[0] = nan(""), acc[1] = nan(""), acc[2] = nan("");
        if (info) atomicCAS(&info->status, 0, (int)ISVD_ERR_INVALID_ARGUMENT);
      }
      continue;
    }
    const float *ui = U + i * ldu;
    const float *vj = V + j * ldv;
    float f = 0.f, a = 0.f, b = 0.f;
    for (int c = lane; c < k; c += 32) {
      const float uv = __ldg(ui + c) * __ldg(vj + c);
      f = fmaf(uv, __ldg(w3 + c), f);
      a = fmaf(uv, __ldg(w3 + k + c), a);
      b = fmaf(uv, __ldg(w3 + 2 * k + c), b);
    }
    const double F = warp_sum((double)f), A = warp_sum((double)a), B = warp_sum((double)b);
    if (lane == 0) {
      // -log sigma(sgn F) = softplus(-sgn F); its derivative in F is -sgn sigma(-sgn F)
      const double sgn = edge ? 1.0 : -1.0;
      const double scale = edge ? pos_scale : neg_scale;
      const double t = -sgn * F;
      const double sp = fmax(t, 0.0) + log1p(exp(-fabs(t)));
      const double g = -sgn * scale / (1.0 + exp(sgn * F));
      acc[0] += scale * sp;
      acc[1] += g * A;
      acc[2] += g * B;
    }
  }
  if (lane == 0) {
    red[warp][0] = acc[0];
    red[warp][1] = acc[1];
    red[warp][2] = acc[2];
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) s += red[wi][threadIdx.x];
    partial[(size_t)blockIdx.x * 3 + threadIdx.x] = s;
  }
}

__global__ void edge_loss_reduce_kernel(const double *__restrict__ partial, int32_t nblocks, double *__restrict__ out) {
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * 3 + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// work layout (doubles): w3 [3k] | w3f [3k floats] | partials [3 x kLossBlocks]
int64_t work_w3f_offset(int32_t k) { return 3 * (int64_t)k; }
int64_t work_partial_offset(int32_t k) { return 3 * (int64_t)k + (3 * (int64_t)k + 1) / 2; }

isvd_status check_factors(const float *U, int64_t ldu, int64_t rows, const float *V, int64_t ldv, int64_t cols,
                          int32_t k, const float *S, const double *work, int64_t work_doubles) {
  if (!U || !V || !S || !work) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  if (k < 1) return fail(ISVD_ERR_SHAPE, "need k >= 1");
  if (rows < 0 || cols < 0) return fail(ISVD_ERR_INVALID_ARGUMENT, "rows and cols must be >= 0");
  if (ldu < k || ldv < k) return fail(ISVD_ERR_INVALID_ARGUMENT, "leading dimension too small");
  if (work_doubles < isvd_edge_kernel_work_doubles(k))
    return fail(ISVD_ERR_INVALID_ARGUMENT, "work holds %lld doubles, %lld needed", (long long)work_doubles,
                (long long)isvd_edge_kernel_work_doubles(k));
  return ISVD_OK;
}

bool finite_params(double mu, double s_bar) { return std::isfinite(mu) && std::isfinite(s_bar); }

}  // namespace
}  // namespace isvd

using namespace isvd;

extern "C" {

int64_t isvd_edge_kernel_work_doubles(int32_t k) {
  if (k < 1) return 0;
  return work_partial_offset(k) + 3 * (int64_t)kLossBlocks;
}

isvd_status isvd_edge_kernel_weights(const float *S, int32_t k, double mu, double s_bar, double *w3, void *stream) {
  if (!S || !w3) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  if (k < 1) return fail(ISVD_ERR_SHAPE, "need k >= 1");
  if (!finite_params(mu, s_bar)) return fail(ISVD_ERR_INVALID_ARGUMENT, "mu and s_bar must be finite");
  edge_weights_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(S, k, mu, s_bar, w3, nullptr);
  ISVD_CUDA_TRY(cudaGetLastError());
  return ISVD_OK;
}

isvd_status isvd_edge_kernel_scores(const float *U, int64_t ldu, int64_t rows, const float *V, int64_t ldv,
                                    int64_t cols, int32_t k, const float *S, double mu, double s_bar,
                                    const int32_t *src, const int32_t *dst, int64_t n_pairs, float *out,
                                    double *work, int64_t work_doubles, isvd_info *dev_info, void *stream) {
  ISVD_TRY(check_factors(U, ldu, rows, V, ldv, cols, k, S, work, work_doubles));
  if (!finite_params(mu, s_bar)) return fail(ISVD_ERR_INVALID_ARGUMENT, "mu and s_bar must be finite");
  if (n_pairs < 0) return fail(ISVD_ERR_INVALID_ARGUMENT, "n_pairs must be >= 0");
  if (n_pairs == 0) return ISVD_OK;
  if (!src || !dst || !out) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  float *w3f = reinterpret_cast<float *>(work + work_w3f_offset(k));
  edge_weights_kernel<<<1, 256, 0, s>>>(S, k, mu, s_bar, work, w3f);
  ISVD_CUDA_TRY(cudaGetLastError());
  const int64_t blocks = std::min<int64_t>(ceil_div(n_pairs, 8), (int64_t)kNumSMs * 8);
  edge_scores_kernel<<<(unsigned)blocks, 256, 0, s>>>(U, ldu, rows, V, ldv, cols, k, w3f, src, dst, n_pairs, out,
                                                      dev_info);
  ISVD_CUDA_TRY(cudaGetLastError());
  return ISVD_OK;
}

isvd_status isvd_edge_kernel_loss(const float *U, int64_t ldu, int64_t rows, const float *V, int64_t ldv,
                                  int64_t cols, int32_t k, const float *S, double mu, double s_bar,
                                  const int32_t *pos_src, const int32_t *pos_dst, int64_t n_pos,
                                  const int32_t *neg_src, const int32_t *neg_dst, int64_t n_neg, double k_neg,
                                  double *out, double *work, int64_t work_doubles, isvd_info *dev_info,
                                  void *stream) {
  ISVD_TRY(check_factors(U, ldu, rows, V, ldv, cols, k, S, work, work_doubles));
  if (!out) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  if (!finite_params(mu, s_bar) || !std::isfinite(k_neg) || k_neg < 0.0)
    return fail(ISVD_ERR_INVALID_ARGUMENT, "mu, s_bar must be finite and k_neg finite and >= 0");
  if (n_pos < 1 || n_neg < 0) return fail(ISVD_ERR_INVALID_ARGUMENT, "need n_pos >= 1 and n_neg >= 0");
  if (!pos_src || !pos_dst || (n_neg > 0 && (!neg_src || !neg_dst)))
    return fail(ISVD_ERR_INVALID_ARGUMENT, "null pair array");
  cudaStream_t s = (cudaStream_t)stream;
  float *w3f = reinterpret_cast<float *>(work + work_w3f_offset(k));
  double *partial = work + work_partial_offset(k);
  edge_weights_kernel<<<1, 256, 0, s>>>(S, k, mu, s_bar, work, w3f);
  ISVD_CUDA_TRY(cudaGetLastError());
  edge_loss_kernel<<<kLossBlocks, 256, 0, s>>>(U, ldu, rows, V, ldv, cols, k, w3f, pos_src, pos_dst, n_pos, neg_src,
                                               neg_dst, n_neg, k_neg, partial, dev_info);
  ISVD_CUDA_TRY(cudaGetLastError());
  edge_loss_reduce_kernel<<<1, 32, 0, s>>>(partial, kLossBlocks, out);
  ISVD_CUDA_TRY(cudaGetLastError());
  return ISVD_OK;
}

}  // extern "C"
