// Closed-form weights from a truncated SVD (Sec. 3, Thm. 1): the least-norm
// minimiser of ||M W - Y||_F is W* = M^+ Y, and with M ~ U S V^T this is
//     W* = V S^+ (U^T Y).
// U^T Y is a tall-skinny transposed product over the r rows of U and Y
// (split over row parts, FP32 products summed per 64-row step, FP64 across
// steps and parts); the k x m result is scaled by S^+ and multiplied into V.
// Also the network-embedding outputs of Sec. 3.1: L = U S^1/2, R = V S^1/2
// and the pair scores f(i, j) = <L_i, R_j>.
#include <algorithm>

#include "internal.h"

namespace isvd {
namespace {

constexpr int kTnRows = 64;  // rows staged in shared memory per step
constexpr int kTnTile = 32;  // output tile (kTnTile x kTnTile) per CTA

// partial[part][i][j] = sum over the part's rows r of A[r][i] B[r][j]
__global__ void __launch_bounds__(256) tn_partial_kernel(const float *__restrict__ A, int64_t lda,
                                                         const float *__restrict__ B, int64_t ldb, int64_t rows,
                                                         int32_t p, int32_t q, int64_t rows_per_part,
                                                         double *__restrict__ partial) {
  __shared__ float As[kTnRows][kTnTile + 1];
  __shared__ float Bs[kTnRows][kTnTile + 1];
  const int tiles_q = (q + kTnTile - 1) / kTnTile;
  const int i0 = (int)(blockIdx.y / tiles_q) * kTnTile, j0 = (int)(blockIdx.y % tiles_q) * kTnTile;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 warps, 4 output rows each
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_part;
  const int64_t r1 = r0 + rows_per_part < rows ? r0 + rows_per_part : rows;
  for (int64_t rb = r0; rb < r1; rb += kTnRows) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kTnRows * kTnTile; idx += blockDim.x) {
      const int rr = idx / kTnTile, c = idx - rr * kTnTile;
      const int64_t r = rb + rr;
      const bool ok = r < r1;
      As[rr][c] = (ok && i0 + c < p) ? A[r * lda + i0 + c] : 0.f;
      Bs[rr][c] = (ok && j0 + c < q) ? B[r * ldb + j0 + c] : 0.f;
    }
    __syncthreads();
    float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
    for (int rr = 0; rr < kTnRows; ++rr) {
      const float b = Bs[rr][tx];
#pragma unroll
      for (int i = 0; i < 4; ++i) s[i] = fmaf(As[rr][ty * 4 + i], b, s[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] += (double)s[i];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int ii = i0 + ty * 4 + i, jj = j0 + tx;
    if (ii < p && jj < q) partial[((size_t)blockIdx.x * p + ii) * q + jj] = acc[i];
  }
}

// Z[i][j] = S^+_i sum_parts partial[part][i][j]; S^+_i = 1/S_i when
// S_i > rcond * max S, else 0.
__global__ void closed_form_reduce_kernel(const double *__restrict__ partial, int32_t nparts, int32_t p, int32_t q,
                                          const float *__restrict__ S, double rcond, float *__restrict__ Z) {
  __shared__ double smax;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < p; ++i) m = fmax(m, (double)S[i]);
    smax = m;
  }
  __syncthreads();
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < p * q; idx += gridDim.x * blockDim.x) {
    const int i = idx / q;
    double t = 0.0;
    for (int pp = 0; pp < nparts; ++pp) t += partial[(size_t)pp * p * q + idx];
    const double si = (double)S[i];
    const double inv = (si > 0.0 && si > rcond * smax) ? 1.0 / si : 0.0;
    Z[idx] = (float)(t * inv);
  }
}

// out = X diag(S)^1/2, one element per thread (grid-stride; out may be X)
__global__ void embed_kernel(const float *X, int64_t ldx, int64_t rows, int32_t k, const float *__restrict__ S,
                             float *out, int64_t ldo) {
  const int64_t total = rows * k;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / k;
    const int j = (int)(idx - r * k);
    out[r * ldo + j] = X[r * ldx + j] * sqrtf(__ldg(S + j));
  }
}

// One warp per pair: lane t multiplies columns t, t + 32, ... in FP32, the
// 32 lane sums are added in FP64 by a butterfly (fixed order).
__global__ void __launch_bounds__(256) pair_scores_kernel(const float *__restrict__ L, int64_t ldl, int64_t rows,
                                                          const float *__restrict__ R, int64_t ldr, int64_t cols,
                                                          int32_t k, const int32_t *__restrict__ src,
                                                          const int32_t *__restrict__ dst, int64_t n_pairs,
                                                          float *__restrict__ out, isvd_info *info) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < n_pairs; p += nwarp) {
    const int64_t i = __ldg(src + p), j = __ldg(dst + p);
    if (i < 0 || i >= rows || j < 0 || j >= cols) {
      if (lane == 0) {
        out[p] = __int_as_float(0x7fc00000);
        if (info) atomicCAS(&info->status, 0, (int)ISVD_ERR_INVALID_ARGUMENT);
      }
      continue;
    }
    const float *li = L + i * ldl;
    const float *rj = R + j * ldr;
    float acc = 0.f;
    for (int c = lane; c < k; c += 32) acc = fmaf(__ldg(li + c), __ldg(rj + c), acc);
    double t = (double)acc;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    if (lane == 0) out[p] = (float)t;
  }
}

}  // namespace

cudaError_t embed_launch(const float *X, int64_t ldx, int64_t rows, int32_t k, const float *S, float *out,
                         int64_t ldo, cudaStream_t s) {
  const int64_t total = rows * k;
  if (total == 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>(ceil_div(total, 256), (int64_t)kNumSMs * 8);
  embed_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, ldx, rows, k, S, out, ldo);
  return cudaGetLastError();
}

cudaError_t pair_scores_launch(const float *L, int64_t ldl, int64_t rows, const float *R, int64_t ldr, int64_t cols,
                               int32_t k, const int32_t *src, const int32_t *dst, int64_t n_pairs, float *out,
                               isvd_info *info, cudaStream_t s) {
  if (n_pairs == 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>(ceil_div(n_pairs, 8), (int64_t)kNumSMs * 8);
  pair_scores_kernel<<<(unsigned)blocks, 256, 0, s>>>(L, ldl, rows, R, ldr, cols, k, src, dst, n_pairs, out, info);
  return cudaGetLastError();
}

int32_t tn_tiles(int32_t p, int32_t q) { return ((p + kTnTile - 1) / kTnTile) * ((q + kTnTile - 1) / kTnTile); }

cudaError_t tn_partial_launch(const float *A, int64_t lda, const float *B, int64_t ldb, int64_t rows, int32_t p,
                              int32_t q, double *partial, int32_t nparts, cudaStream_t s) {
  const int64_t rpp = round_up(ceil_div(rows, nparts), kTnRows);
  tn_partial_kernel<<<dim3((unsigned)nparts, (unsigned)tn_tiles(p, q)), 256, 0, s>>>(A, lda, B, ldb, rows, p, q, rpp,
                                                                                      partial);
  return cudaGetLastError();
}

int32_t closed_form_parts(int64_t rows, int32_t k, int32_t m) {
  const int tiles = ((k + kTnTile - 1) / kTnTile) * ((m + kTnTile - 1) / kTnTile);
  int64_t parts = ceil_div(rows, 1024);
  const int64_t cap = (2 * kNumSMs + tiles - 1) / tiles;
  if (parts > cap) parts = cap;
  if (parts < 1) parts = 1;
  // room for the tensor-core form's partial count too
  return std::max<int32_t>((int32_t)parts, gram_ab_parts(rows));
}

// U^T Y on the tensor cores (k <= 128, m <= 160) or the CUDA cores, then
// Z = diag(S)^+ (U^T Y), then W = V Z on the tensor cores where the layout
// suits them.  nparts: the capacity of `partial` (closed_form_parts).
cudaError_t closed_form_launch(const float *U, int64_t ldu, const float *S, const float *V, int64_t ldv, int64_t r,
                               int64_t c, int32_t k, const float *Y, int64_t ldy, int32_t m, double rcond,
                               float *W, int64_t ldw, double *partial, int32_t nparts, float *Z, cudaStream_t s) {
  bool tc = false;
  int32_t used = std::min(nparts, gram_ab_parts(r));
  cudaError_t e = gram_ab_launch(U, ldu, k, Y, ldy, m, r, partial, used, nullptr, &tc, s);
  if (e != cudaSuccess) return e;
  if (!tc) {
    const int tiles = ((k + kTnTile - 1) / kTnTile) * ((m + kTnTile - 1) / kTnTile);
    used = nparts;
    const int64_t rpp = round_up(ceil_div(r, used), kTnRows);
    tn_partial_kernel<<<dim3((unsigned)used, (unsigned)tiles), 256, 0, s>>>(U, ldu, Y, ldy, r, k, m, rpp, partial);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  closed_form_reduce_kernel<<<(unsigned)ceil_div((int64_t)k * m, 256), 256, 0, s>>>(partial, used, k, m, S, rcond, Z);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  bool launched = false;
  e = gemm_tc_launch(V, ldv, c, k, Z, m, m, W, ldw, &launched, s);
  if (e != cudaSuccess || launched) return e;
  return gemm_small_launch(V, ldv, DT_F32, c, k, Z, m, m, false, W, ldw, DT_F32, PassGate{}, s);
}

}  // namespace isvd
