// Closed-form weights from a truncated SVD (Sec. 3, Thm. 1): the least-norm
// minimiser of ||M W - Y||_F is W* = M^+ Y, and with M ~ U S V^T this is
//     W* = V S^+ (U^T Y).
// U^T Y is a tall-skinny transposed product over the r rows of U and Y
// (split over row parts, FP32 products summed per 64-row step, FP64 across
// steps and parts); the k x m result is scaled by S^+ and multiplied into V.
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

}  // namespace

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
  return (int32_t)parts;
}

cudaError_t closed_form_launch(const float *U, int64_t ldu, const float *S, const float *V, int64_t ldv, int64_t r,
                               int64_t c, int32_t k, const float *Y, int64_t ldy, int32_t m, double rcond,
                               float *W, int64_t ldw, double *partial, int32_t nparts, float *Z, cudaStream_t s) {
  const int tiles = ((k + kTnTile - 1) / kTnTile) * ((m + kTnTile - 1) / kTnTile);
  const int64_t rpp = round_up(ceil_div(r, nparts), kTnRows);
  tn_partial_kernel<<<dim3((unsigned)nparts, (unsigned)tiles), 256, 0, s>>>(U, ldu, Y, ldy, r, k, m, rpp, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  closed_form_reduce_kernel<<<(unsigned)ceil_div((int64_t)k * m, 256), 256, 0, s>>>(partial, nparts, k, m, S, rcond,
                                                                                   Z);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return gemm_small_launch(V, ldv, DT_F32, c, k, Z, m, m, false, W, ldw, DT_F32, PassGate{}, s);
}

}  // namespace isvd
