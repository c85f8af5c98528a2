// Dense helpers of the randomized SVD: the Gaussian start block (Alg. 1),
// V^T G projections for the rank-one / low-rank corrections (Eq. 3's
// all-ones term), the Gram matrix Q^T Q and the block-times-small-matrix
// product Q B of CholeskyQR (Alg. 2) and of the Rayleigh-Ritz step.
#include <mutex>

#include "internal.h"
#include "philox.cuh"

namespace isvd {
namespace {

template <typename T>
__device__ __forceinline__ T from_float(float x);
template <>
__device__ __forceinline__ float from_float<float>(float x) { return x; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_float<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

__device__ __forceinline__ float to_float(float x) { return x; }
__device__ __forceinline__ float to_float(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename T>
__global__ void gaussian_kernel(uint32_t k0, uint32_t k1, int64_t rows, int32_t cols, T *out, int64_t ld) {
  const int64_t nq = ld / 4;
  const int64_t total = rows * nq;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / nq;
    const int32_t q = (int32_t)(idx - i * nq);
    float z[4] = {0.f, 0.f, 0.f, 0.f};
    if (4 * q < cols) gaussian_quad(k0, k1, i, q, z);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int c = 4 * q + t;
      out[i * ld + c] = from_float<T>(c < cols ? z[t] : 0.f);
    }
  }
}

__global__ void philox_words_kernel(uint32_t k0, uint32_t k1, int64_t rows, uint32_t *out) {
  const int64_t total = rows * 4;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / 4;
    const uint32_t j = (uint32_t)(idx & 3);
    uint32_t c0 = j, c1 = (uint32_t)i, c2 = (uint32_t)((uint64_t)i >> 32), c3 = 0u;
    philox4x32_10(c0, c1, c2, c3, k0, k1);
    uint32_t *o = out + i * 16 + 4 * j;
    o[0] = c0;
    o[1] = c1;
    o[2] = c2;
    o[3] = c3;
  }
}

// ---- V^T G, deterministic two-phase reduction ----------------------------------
// Phase 1: block p sums rows p*8+y, step n_part*8, in FP32 per thread (4
// columns each), then the 8 row lanes are combined in FP64.  Phase 2 adds the
// n_part partials in block order in FP64.
template <typename T>
__device__ __forceinline__ void load4(const T *p, float *v);
template <>
__device__ __forceinline__ void load4<float>(const float *p, float *v) {
  const float4 x = *reinterpret_cast<const float4 *>(p);
  v[0] = x.x;
  v[1] = x.y;
  v[2] = x.z;
  v[3] = x.w;
}
template <>
__device__ __forceinline__ void load4<__nv_bfloat16>(const __nv_bfloat16 *p, float *v) {
  const uint2 x = *reinterpret_cast<const uint2 *>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&x.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&x.y));
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

// Lane x of a warp owns columns [4x, 4x + 4) and [128 + 4x, 132 + 4x) of each
// 256-column pass (one vector load each; columns past b are loaded from the
// row's padding, which ld % 8 == 0 keeps inside the row, and not summed).
template <typename T, int RMAX>
__global__ void __launch_bounds__(256) project_partial_kernel(const T *G, int64_t ldg, int64_t rows, int32_t b,
                                                              const float *V, int64_t ldv, int32_t r,
                                                              int32_t ones_first, double *partial, int64_t pb) {
  __shared__ double red[8][33];
  const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
  const int64_t p = blockIdx.x;
  const int64_t stride = (int64_t)gridDim.x * 8;
  for (int c0 = 0; c0 < b; c0 += 256) {
    const int colA = c0 + 4 * x, colB = c0 + 128 + 4 * x;
    const bool inA = colA < b, inB = colB < b;
    float acc[RMAX][8];
#pragma unroll
    for (int t = 0; t < RMAX; ++t)
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[t][k] = 0.f;
    if (inA) {
      // unrolled: the loads of four rows are in flight together (the sums keep their order)
#pragma unroll 4
      for (int64_t i = p * 8 + y; i < rows; i += stride) {
        float v[8];
        load4<T>(G + i * ldg + colA, v);
        if (inB) load4<T>(G + i * ldg + colB, v + 4);
        else v[4] = v[5] = v[6] = v[7] = 0.f;
#pragma unroll
        for (int t = 0; t < RMAX; ++t) {
          if (t < r) {
            const int tv = t - ones_first;
            const float u = (tv < 0 || !V) ? 1.f : V[i * ldv + tv];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[t][k] = fmaf(u, v[k], acc[t][k]);
          }
        }
      }
    }
    // sum the 8 row warps, one column at a time, in FP64
#pragma unroll
    for (int t = 0; t < RMAX; ++t) {
      if (t >= r) break;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        red[y][x] = (double)acc[t][k];
        __syncthreads();
        if (y == 0) {
          double sacc = 0.0;
          for (int yy = 0; yy < 8; ++yy) sacc += red[yy][x];
          const int col = (k < 4 ? colA : colB) + (k & 3);
          if (col < b && (k < 4 ? inA : inB)) partial[(p * r + t) * pb + col] = sacc;
        }
        __syncthreads();
      }
    }
  }
}

// one warp per output: lane j sums partials j, j + 32, ... in order, then a
// fixed shuffle tree (the same order on every run)
__global__ void project_final_kernel(const double *partial, int32_t n_part, int32_t r, int32_t b, int64_t pb,
                                     float *c, int64_t ldc) {
  const int64_t idx = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (idx >= (int64_t)r * b) return;  // uniform within the warp
  const int t = (int)(idx / b), col = (int)(idx % b);
  double s = 0.0;
  for (int p = lane; p < n_part; p += 32) s += partial[((int64_t)p * r + t) * pb + col];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) c[(int64_t)t * ldc + col] = (float)s;
}

// ---- conditional CholeskyQR passes ------------------------------------------------
__device__ __forceinline__ bool pass_skipped(const PassGate &g) {
  return g.state != nullptr && g.pass > 2 && g.state[0] + 2 < g.pass;
}

// ---- out = Q B  (B small, staged in shared memory) -------------------------------
constexpr int kGemmRows = 32;

template <typename TI, typename TO>
__global__ void __launch_bounds__(256) gemm_small_kernel(const TI *Q, int64_t ldq, int64_t rows, int32_t l,
                                                         const float *B, int64_t ldb, int32_t w, int32_t upper,
                                                         TO *out, int64_t ldo, PassGate g) {
  if (pass_skipped(g)) return;
  extern __shared__ float sm[];
  const int wp = (w + 31) / 32 * 32;
  float *Bs = sm;               // [l][wp]
  float *Qs = sm + l * wp;      // [kGemmRows][l]
  for (int idx = threadIdx.x; idx < l * wp; idx += blockDim.x) {
    const int t = idx / wp, c = idx - t * wp;
    Bs[idx] = (c < w && (!upper || c >= t)) ? B[t * ldb + c] : 0.f;
  }
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int nm = wp / 32;
  for (int64_t rt = (int64_t)blockIdx.x * kGemmRows; rt < rows; rt += (int64_t)gridDim.x * kGemmRows) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kGemmRows * l; idx += blockDim.x) {
      const int rr = idx / l, c = idx - rr * l;
      Qs[idx] = (rt + rr < rows) ? to_float(Q[(rt + rr) * ldq + c]) : 0.f;
    }
    __syncthreads();
    float acc[4][5];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int m = 0; m < 5; ++m) acc[i][m] = 0.f;
    for (int t = 0; t < l; ++t) {
      float a[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Qs[(ty * 4 + i) * l + t];
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        if (m < nm) {
          const float bb = Bs[t * wp + tx + 32 * m];
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[i][m] = fmaf(a[i], bb, acc[i][m]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t row = rt + ty * 4 + i;
      if (row >= rows) continue;
#pragma unroll
      for (int m = 0; m < 5; ++m) {
        const int c = tx + 32 * m;
        if (m < nm && c < w) out[row * ldo + c] = from_float<TO>(acc[i][m]);
      }
    }
  }
}

size_t gemm_smem(int32_t l, int32_t w) {
  const int wp = (w + 31) / 32 * 32;
  return sizeof(float) * ((size_t)l * wp + (size_t)kGemmRows * l);
}

// the kernel's shared-memory limit: a 160 x 160 B, or 64 columns of a 512-row B
size_t gemm_smem_cap() {
  const size_t a = gemm_smem(ISVD_MAX_BLOCK, ISVD_MAX_BLOCK), b = gemm_smem(ISVD_MAX_BLOCK_WIDE, 64);
  return a > b ? a : b;
}

// Column slices of at most 160 (five accumulators a lane) whose B fits the
// shared memory; an in-place (upper) product must fit in one.
template <typename TI, typename TO>
cudaError_t gemm_small_t(const void *Q, int64_t ldq, int64_t rows, int32_t l, const float *B, int64_t ldb,
                         int32_t w, bool upper, void *out, int64_t ldo, PassGate g, cudaStream_t s) {
  int64_t bx = ceil_div(rows, kGemmRows);
  if (bx > kNumSMs * 2) bx = kNumSMs * 2;
  if (bx < 1) bx = 1;
  int32_t ws = w < ISVD_MAX_BLOCK ? w : ISVD_MAX_BLOCK;
  while (ws > 32 && gemm_smem(l, ws) > gemm_smem_cap()) ws = (ws - 1) / 32 * 32;
  if (gemm_smem(l, ws) > gemm_smem_cap() || (upper && ws < w)) return cudaErrorInvalidValue;
  for (int32_t c0 = 0; c0 < w; c0 += ws) {
    const int32_t wc = w - c0 < ws ? w - c0 : ws;
    gemm_small_kernel<TI, TO><<<(unsigned)bx, 256, gemm_smem(l, wc), s>>>(
        (const TI *)Q, ldq, rows, l, B + c0, ldb, wc, upper ? 1 : 0, (TO *)out + c0, ldo, g);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t dense_kernels_init() {
  static cudaError_t err = cudaSuccess;
  static std::once_flag once;
  std::call_once(once, [] {
    const int big = (int)gemm_smem_cap();
    cudaError_t e = cudaSuccess;
    e = cudaFuncSetAttribute(gemm_small_kernel<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gemm_small_kernel<__nv_bfloat16, __nv_bfloat16>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gemm_small_kernel<__nv_bfloat16, float>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gemm_small_kernel<float, __nv_bfloat16>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    err = e;
  });
  return err;
}

cudaError_t gaussian_launch(uint64_t seed, int64_t rows, int32_t cols, void *out, int64_t ld, int dtype,
                            cudaStream_t s) {
  const int64_t total = rows * (ld / 4);
  if (total == 0) return cudaSuccess;
  int64_t blocks = ceil_div(total, 256);
  if (blocks > kNumSMs * 32) blocks = kNumSMs * 32;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  if (dtype == DT_F32)
    gaussian_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(k0, k1, rows, cols, (float *)out, ld);
  else
    gaussian_kernel<__nv_bfloat16><<<(unsigned)blocks, 256, 0, s>>>(k0, k1, rows, cols, (__nv_bfloat16 *)out, ld);
  return cudaGetLastError();
}

cudaError_t philox_words_launch(uint64_t seed, int64_t rows, uint32_t *out, cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  int64_t blocks = ceil_div(rows * 4, 256);
  if (blocks > kNumSMs * 32) blocks = kNumSMs * 32;
  philox_words_kernel<<<(unsigned)blocks, 256, 0, s>>>((uint32_t)seed, (uint32_t)(seed >> 32), rows, out);
  return cudaGetLastError();
}

int32_t lowrank_partials(int64_t rows) {
  int64_t p = ceil_div(rows, 256);
  if (p > 512) p = 512;
  if (p < 1) p = 1;
  return (int32_t)p;
}

cudaError_t lowrank_project_launch(const void *G, int64_t ldg, int dtype, int64_t rows, int32_t b, const float *V,
                                   int64_t ldv, int32_t r, int32_t ones_first, double *partial, int32_t n_part,
                                   float *c, int64_t ldc, cudaStream_t s) {
  const int64_t pb = round_up(b, 8);
  // the all-ones projection alone (r = 1) keeps one accumulator row: more resident warps
  if (dtype == DT_F32) {
    if (r == 1)
      project_partial_kernel<float, 1><<<n_part, 256, 0, s>>>((const float *)G, ldg, rows, b, V, ldv, r, ones_first,
                                                               partial, pb);
    else
      project_partial_kernel<float, ISVD_MAX_LOWRANK><<<n_part, 256, 0, s>>>((const float *)G, ldg, rows, b, V, ldv, r,
                                                                              ones_first, partial, pb);
  } else {
    if (r == 1)
      project_partial_kernel<__nv_bfloat16, 1><<<n_part, 256, 0, s>>>((const __nv_bfloat16 *)G, ldg, rows, b, V, ldv,
                                                                       r, ones_first, partial, pb);
    else
      project_partial_kernel<__nv_bfloat16, ISVD_MAX_LOWRANK><<<n_part, 256, 0, s>>>(
          (const __nv_bfloat16 *)G, ldg, rows, b, V, ldv, r, ones_first, partial, pb);
  }
  const int64_t tot = (int64_t)r * b;
  project_final_kernel<<<(unsigned)ceil_div(tot * 32, 256), 256, 0, s>>>(partial, n_part, r, b, pb, c, ldc);
  return cudaGetLastError();
}

cudaError_t gemm_small_launch(const void *Q, int64_t ldq, int in_dtype, int64_t rows, int32_t l, const float *B,
                              int64_t ldb, int32_t w, bool upper, void *out, int64_t ldo, int out_dtype, PassGate g,
                              cudaStream_t s) {
  if (rows == 0) return cudaSuccess;
  if (in_dtype == DT_F32 && out_dtype == DT_F32)
    return gemm_small_t<float, float>(Q, ldq, rows, l, B, ldb, w, upper, out, ldo, g, s);
  if (in_dtype == DT_BF16 && out_dtype == DT_BF16)
    return gemm_small_t<__nv_bfloat16, __nv_bfloat16>(Q, ldq, rows, l, B, ldb, w, upper, out, ldo, g, s);
  if (in_dtype == DT_BF16 && out_dtype == DT_F32)
    return gemm_small_t<__nv_bfloat16, float>(Q, ldq, rows, l, B, ldb, w, upper, out, ldo, g, s);
  return gemm_small_t<float, __nv_bfloat16>(Q, ldq, rows, l, B, ldb, w, upper, out, ldo, g, s);
}

}  // namespace isvd
