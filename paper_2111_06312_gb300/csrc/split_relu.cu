// Split-ReLU layer of the fine-tuning network (Sec. 5.2):
//     Z = [X Wp]_+ - [X Wn]_+
// with X n x d and Wp, Wn d x e.  With Wp = I, Wn = -I (the start from the
// closed-form solution) the layer is the identity (relu(t) - relu(-t) = t),
// which makes the network equal the linear model of Eq. 6 (Thm. 2).
//
// Forward: the pre-activations Ap = X Wp and An = X Wn on the tensor cores
// (the Q.B kernel, 3xTF32), then one elementwise pass for Z.  Backward, with
// Gp = dZ * 1[Ap > 0] and Gn = -dZ * 1[An > 0]:
//     dWp = X^T Gp, dWn = X^T Gn   (the tcgen05 A^T B kernel, FP64 partials)
//     dX  = Gp Wp^T + Gn Wn^T      (the Q.B kernel twice, summed)
// The CUDA-core small-matrix products stand in where a layout does not suit
// the tensor-core kernels.
#include <algorithm>

#include "internal.h"

namespace isvd {
namespace {

int grid_for_elems(int64_t n) {
  int64_t g = ceil_div(n, 256);
  if (g > (int64_t)kNumSMs * 16) g = (int64_t)kNumSMs * 16;
  return (int)(g < 1 ? 1 : g);
}

// Z = relu(Ap) - relu(An)
__global__ void split_relu_fwd_kernel(const float *__restrict__ Ap, const float *__restrict__ An, int64_t lda,
                                      int64_t n, int32_t e, float *__restrict__ Z, int64_t ldz) {
  const int64_t total = n * e;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / e;
    const int c = (int)(idx - i * e);
    const float a = Ap[i * lda + c], b = An[i * lda + c];
    Z[i * ldz + c] = fmaxf(a, 0.f) - fmaxf(b, 0.f);
  }
}

// Gp = dZ * 1[Ap > 0], Gn = -dZ * 1[An > 0] (padding columns zero)
__global__ void split_relu_mask_kernel(const float *__restrict__ Ap, const float *__restrict__ An, int64_t lda,
                                       const float *__restrict__ dZ, int64_t ldz, int64_t n, int32_t e, int32_t ldg,
                                       float *__restrict__ Gp, float *__restrict__ Gn) {
  const int64_t total = n * ldg;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / ldg;
    const int c = (int)(idx - i * ldg);
    float gp = 0.f, gn = 0.f;
    if (c < e) {
      const float g = dZ[i * ldz + c];
      gp = Ap[i * lda + c] > 0.f ? g : 0.f;
      gn = An[i * lda + c] > 0.f ? -g : 0.f;
    }
    Gp[idx] = gp;
    Gn[idx] = gn;
  }
}

// WT (e x d, ld ldt) = W^T for W d x e (ld e)
__global__ void transpose_kernel(const float *__restrict__ W, int32_t d, int32_t e, float *__restrict__ WT,
                                 int32_t ldt) {
  const int total = e * ldt;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    const int c = idx / ldt, r = idx - c * ldt;
    WT[idx] = r < d ? W[(int64_t)r * e + c] : 0.f;
  }
}

// dW (d x e, ld e) = sum over parts of partial[part][r][c] (FP64, fixed order)
__global__ void sum_partials_kernel(const double *__restrict__ partial, int32_t parts, int32_t d, int32_t e,
                                    float *__restrict__ dW) {
  const int total = d * e;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < parts; ++p) s += partial[(size_t)p * total + idx];
    dW[idx] = (float)s;
  }
}

// Y += X (n x d blocks)
__global__ void add_block_kernel(const float *__restrict__ X, int64_t ldx, float *__restrict__ Y, int64_t ldy,
                                 int64_t n, int32_t d) {
  const int64_t total = n * d;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / d;
    const int c = (int)(idx - i * d);
    Y[i * ldy + c] += X[i * ldx + c];
  }
}

// out (n x w) = Q (n x l) B (l x w): tensor cores where they fit, else CUDA cores
cudaError_t product(const float *Q, int64_t ldq, int64_t n, int32_t l, const float *B, int64_t ldb, int32_t w,
                    float *out, int64_t ldo, cudaStream_t s) {
  bool launched = false;
  cudaError_t e = gemm_tc_launch(Q, ldq, n, l, B, ldb, w, out, ldo, &launched, s);
  if (e != cudaSuccess || launched) return e;
  return gemm_small_launch(Q, ldq, DT_F32, n, l, B, ldb, w, false, out, ldo, DT_F32, PassGate{}, s);
}

struct Work {
  float *Gp, *Gn, *WpT, *WnT, *T2;
  double *partial;
  int32_t parts, ldg, ldt;
};

size_t carve(int64_t n, int32_t d, int32_t e, char *base, Work *w) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char *p = base ? base + off : nullptr;
    off += (size_t)round_up((int64_t)bytes, 256);
    return p;
  };
  Work x{};
  x.ldg = (int32_t)round_up(e, 4);
  x.ldt = (int32_t)round_up(d, 4);
  x.parts = gram_ab_parts(n);  // row ranges of X^T G, for either kernel
  x.Gp = (float *)take(sizeof(float) * (size_t)n * x.ldg);
  x.Gn = (float *)take(sizeof(float) * (size_t)n * x.ldg);
  x.WpT = (float *)take(sizeof(float) * (size_t)e * x.ldt);
  x.WnT = (float *)take(sizeof(float) * (size_t)e * x.ldt);
  x.T2 = (float *)take(sizeof(float) * (size_t)n * x.ldt);
  x.partial = (double *)take(sizeof(double) * (size_t)x.parts * d * e);
  if (w) *w = x;
  return off;
}

// C (d x e, FP32, ld e) = X^T G over n rows
cudaError_t xt_g(const float *X, int64_t ldx, int64_t n, int32_t d, const float *G, int64_t ldg, int32_t e,
                 const Work &w, float *C, cudaStream_t s) {
  bool tc = false;
  cudaError_t err = gram_ab_launch(X, ldx, d, G, ldg, e, n, w.partial, w.parts, nullptr, &tc, s);
  if (err != cudaSuccess) return err;
  if (!tc) {
    err = tn_partial_launch(X, ldx, G, ldg, n, d, e, w.partial, w.parts, s);
    if (err != cudaSuccess) return err;
  }
  sum_partials_kernel<<<grid_for_elems((int64_t)d * e), 256, 0, s>>>(w.partial, w.parts, d, e, C);
  return cudaGetLastError();
}

}  // namespace
}  // namespace isvd

using namespace isvd;

extern "C" {

size_t isvd_split_relu_work_bytes(int64_t n, int32_t d, int32_t e) {
  if (n < 1 || d < 1 || e < 1) return 0;
  return carve(n, d, e, nullptr, nullptr);
}

isvd_status isvd_split_relu_forward(const float *X, int64_t ldx, int64_t n, int32_t d, const float *Wp,
                                    const float *Wn, int32_t e, float *Z, int64_t ldz, float *Ap, float *An,
                                    int64_t lda, void *stream) {
  if (!X || !Wp || !Wn || !Z || !Ap || !An) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  if (n < 1 || d < 1 || e < 1 || d > ISVD_MAX_BLOCK || e > ISVD_MAX_BLOCK)
    return fail(ISVD_ERR_SHAPE, "need n >= 1 and 1 <= d, e <= %d", ISVD_MAX_BLOCK);
  if (ldx < d || ldz < e || lda < e) return fail(ISVD_ERR_INVALID_ARGUMENT, "leading dimension too small");
  cudaStream_t s = (cudaStream_t)stream;
  ISVD_CUDA_TRY(product(X, ldx, n, d, Wp, e, e, Ap, lda, s));
  ISVD_CUDA_TRY(product(X, ldx, n, d, Wn, e, e, An, lda, s));
  split_relu_fwd_kernel<<<grid_for_elems(n * e), 256, 0, s>>>(Ap, An, lda, n, e, Z, ldz);
  ISVD_CUDA_TRY(cudaGetLastError());
  return ISVD_OK;
}

isvd_status isvd_split_relu_backward(const float *X, int64_t ldx, int64_t n, int32_t d, const float *Wp,
                                     const float *Wn, int32_t e, const float *Ap, const float *An, int64_t lda,
                                     const float *dZ, int64_t ldz, float *dX, int64_t lddx, float *dWp, float *dWn,
                                     void *work, size_t work_bytes, void *stream) {
  if (!X || !Wp || !Wn || !Ap || !An || !dZ || !dWp || !dWn || !work)
    return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  if (n < 1 || d < 1 || e < 1 || d > ISVD_MAX_BLOCK || e > ISVD_MAX_BLOCK)
    return fail(ISVD_ERR_SHAPE, "need n >= 1 and 1 <= d, e <= %d", ISVD_MAX_BLOCK);
  if (ldx < d || ldz < e || lda < e || (dX && lddx < d))
    return fail(ISVD_ERR_INVALID_ARGUMENT, "leading dimension too small");
  if (work_bytes < isvd_split_relu_work_bytes(n, d, e) || ((uintptr_t)work & 255))
    return fail(ISVD_ERR_WORKSPACE, "work must be 256-byte aligned and hold isvd_split_relu_work_bytes(n, d, e)");
  cudaStream_t s = (cudaStream_t)stream;
  Work w;
  carve(n, d, e, (char *)work, &w);
  split_relu_mask_kernel<<<grid_for_elems(n * w.ldg), 256, 0, s>>>(Ap, An, lda, dZ, ldz, n, e, w.ldg, w.Gp, w.Gn);
  ISVD_CUDA_TRY(cudaGetLastError());
  ISVD_CUDA_TRY(xt_g(X, ldx, n, d, w.Gp, w.ldg, e, w, dWp, s));
  ISVD_CUDA_TRY(xt_g(X, ldx, n, d, w.Gn, w.ldg, e, w, dWn, s));
  if (dX) {
    transpose_kernel<<<grid_for_elems((int64_t)e * w.ldt), 256, 0, s>>>(Wp, d, e, w.WpT, w.ldt);
    transpose_kernel<<<grid_for_elems((int64_t)e * w.ldt), 256, 0, s>>>(Wn, d, e, w.WnT, w.ldt);
    ISVD_CUDA_TRY(cudaGetLastError());
    ISVD_CUDA_TRY(product(w.Gp, w.ldg, n, e, w.WpT, w.ldt, d, dX, lddx, s));
    ISVD_CUDA_TRY(product(w.Gn, w.ldg, n, e, w.WnT, w.ldt, d, w.T2, w.ldt, s));
    add_block_kernel<<<grid_for_elems(n * d), 256, 0, s>>>(w.T2, w.ldt, dX, lddx, n, d);
    ISVD_CUDA_TRY(cudaGetLastError());
  }
  return ISVD_OK;
}

}  // extern "C"
