// Dense feature matrices in the CONCAT operator M = [X | N X | ... | N^L X]
// (Eq. 6).  With X dense (n x d, FP32), the products with X are small dense
// matrix products rather than sparse ones:
//   forward   P = X [G_0 | ... | G_L]       (n x d times d x (L+1) b, one pass over X)
//   transpose out_l = X^T P_l, stacked       (d x n times n x (L+1) b, split over rows)
// The forward product restacks the (L+1) d x b input blocks side by side
// (FP32) and runs X B on the tensor cores (the Q.B kernel that closes Alg. 1;
// the CUDA-core small-matrix product for BF16 output or unsuitable layouts);
// the transposed product takes X^T P on the tensor cores (A^T B with FP64
// partials per row range, added in a fixed order) and writes each d x b
// segment to its place in the (L+1) d x b output.
#include <algorithm>

#include "internal.h"

namespace isvd {
namespace {

template <typename T>
__device__ __forceinline__ float ld_as_float(const T *p);
template <>
__device__ __forceinline__ float ld_as_float<float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float ld_as_float<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// B[t][l * bseg + c] = G[(l d + t) ldg + c] (c < b), 0 in the padding columns
template <typename T>
__global__ void restack_kernel(const T *__restrict__ G, int64_t ldg, int32_t d, int32_t b, int32_t bseg,
                               int32_t segs, float *__restrict__ B) {
  const int64_t total = (int64_t)d * segs * bseg;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = idx / (segs * bseg);
    const int rem = (int)(idx - t * segs * bseg);
    const int l = rem / bseg, c = rem - l * bseg;
    B[idx] = c < b ? ld_as_float(G + ((size_t)l * d + t) * ldg + c) : 0.f;
  }
}

// rows [0, n) of block `src` (width b) into the first b columns of `dst`
__global__ void copy_cols_kernel(const float *__restrict__ src, int64_t lds, float *__restrict__ dst, int64_t ldd,
                                 int64_t n, int32_t b) {
  const int64_t total = n * b;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / b;
    const int c = (int)(idx - i * b);
    dst[i * ldd + c] = src[i * lds + c];
  }
}

// out[(l d + t) ldo + c] = sum_parts partial[part][t][l bseg + c]
__global__ void tn_reduce_stacked_kernel(const double *__restrict__ partial, int32_t nparts, int32_t d, int32_t q,
                                         int32_t b, int32_t bseg, float *__restrict__ out, int64_t ldo) {
  const int total = d * q;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int t = idx / q, col = idx - t * q;
    const int l = col / bseg, c = col - l * bseg;
    if (c >= b) continue;
    double s = 0.0;
    for (int pp = 0; pp < nparts; ++pp) s += partial[(size_t)pp * d * q + idx];
    out[((size_t)l * d + t) * ldo + c] = (float)s;
  }
}

int grid_for(int64_t n) {
  int64_t g = ceil_div(n, 256);
  if (g > kNumSMs * 16) g = kNumSMs * 16;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

size_t xdense_scratch_bytes(int32_t d, int32_t segs, int32_t bseg, int64_t n) {
  const int32_t q = segs * bseg;
  const int32_t parts = std::max(xdense_parts(n, d, q), gram_ab_parts(n));
  return (size_t)round_up((int64_t)sizeof(float) * d * q, 256) + (size_t)round_up((int64_t)sizeof(double) * parts * d * q, 256);
}

int32_t xdense_parts(int64_t n, int32_t d, int32_t q) {
  int64_t parts = ceil_div(n, 2048);
  const int64_t cap = (2 * kNumSMs + tn_tiles(d, q) - 1) / tn_tiles(d, q);
  if (parts > cap) parts = cap;
  if (parts < 1) parts = 1;
  return (int32_t)parts;
}

cudaError_t xdense_forward(const float *X, int64_t n, int32_t d, const void *G, int64_t ldg, int dtype, int32_t b,
                           int32_t bseg, int32_t segs, void *P, int64_t ldp, void *scratch, cudaStream_t s) {
  float *B = reinterpret_cast<float *>(scratch);
  const int64_t tot = (int64_t)d * segs * bseg;
  if (dtype == DT_F32)
    restack_kernel<float><<<grid_for(tot), 256, 0, s>>>((const float *)G, ldg, d, b, bseg, segs, B);
  else
    restack_kernel<__nv_bfloat16><<<grid_for(tot), 256, 0, s>>>((const __nv_bfloat16 *)G, ldg, d, b, bseg, segs, B);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // all (L+1) segments, padding columns included (zero), in one pass over X;
  // a single segment is the caller's block: its b columns only.  FP32 on the
  // tensor cores (3xTF32) where the layout suits them
  const int32_t w = segs == 1 ? b : segs * bseg;
  if (dtype == DT_F32) {
    bool launched = false;
    e = gemm_tc_launch(X, d, n, d, B, (int64_t)segs * bseg, w, reinterpret_cast<float *>(P), ldp, &launched, s);
    if (e != cudaSuccess || launched) return e;
  }
  return gemm_small_launch(X, d, DT_F32, n, d, B, (int64_t)segs * bseg, w, false, P, ldp, dtype, PassGate{}, s);
}

cudaError_t xdense_transpose(const float *X, int64_t n, int32_t d, const float *H, int64_t ldh, int32_t b,
                             int32_t bseg, int32_t segs, float *P, int64_t ldp, float *out, int64_t ldo, void *scratch,
                             cudaStream_t s) {
  const int32_t q = segs * bseg;
  double *partial = reinterpret_cast<double *>(reinterpret_cast<char *>(scratch) +
                                               round_up((int64_t)sizeof(float) * d * q, 256));
  // segment 0 of P holds H itself
  copy_cols_kernel<<<grid_for(n * b), 256, 0, s>>>(H, ldh, P, ldp, n, b);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // X^T P on the tensor cores where the shapes suit them (d <= 128, q <= 160)
  bool tc = false;
  int32_t parts = gram_ab_parts(n);
  e = gram_ab_launch(X, d, d, P, ldp, q, n, partial, parts, nullptr, &tc, s);
  if (e != cudaSuccess) return e;
  if (!tc) {
    parts = xdense_parts(n, d, q);
    e = tn_partial_launch(X, d, P, ldp, n, d, q, partial, parts, s);
    if (e != cudaSuccess) return e;
  }
  tn_reduce_stacked_kernel<<<(unsigned)ceil_div((int64_t)d * q, 256), 256, 0, s>>>(partial, parts, d, q, b, bseg, out,
                                                                                  ldo);
  return cudaGetLastError();
}

}  // namespace isvd
