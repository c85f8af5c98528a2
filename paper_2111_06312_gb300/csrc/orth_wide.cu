// Orthonormalisation of a wide block (128 < l <= 512 columns, FP32) for Alg. 1
// at the paper's own block widths (rank 250 or 256 with 2k columns, Sec. 6).
//
// The Gram matrix of a 512-column block does not fit the CholeskyQR kernels
// (one 128 x 160 tile pair of tensor memory, one cluster's shared memory for
// the FP64 factor), so the block is taken in panels of 128 columns, left to
// right, by block Gram-Schmidt with reorthogonalisation (BCGS2): panel j is
// projected off the panels before it twice,
//     C = Q_<j^T Y,  Y <- Y - Q_<j C      (C summed in FP64 over row ranges)
// and then orthonormalised by CholeskyQR2 (Alg. 2, twice, with the shift on
// breakdown); the subtraction happens in the epilogue of the Q_i C product.  The result is the thin QR of the block (the same Q and R, up
// to rounding, as one CholeskyQR2 of all l columns): R is block upper
// triangular with the two projections' C above the diagonal and the panels'
// CholeskyQR factors on it.  Q_i^T Y runs on the tcgen05 A^T B kernel,
// Q_i C on the Q.B kernel.
#include <algorithm>

#include "internal.h"

namespace isvd {
namespace {

constexpr int32_t kPanel = 128;

int grid_for_elems(int64_t n) {
  int64_t g = ceil_div(n, 256);
  if (g > (int64_t)kNumSMs * 16) g = (int64_t)kNumSMs * 16;
  return (int)(g < 1 ? 1 : g);
}

// C32 (p x q, ld q) = sum over parts of partial[part][r][c]; Racc block += it
__global__ void wide_reduce_kernel(const double *__restrict__ partial, int32_t parts, int32_t p, int32_t q,
                                   float *__restrict__ C32, double *__restrict__ Racc, int32_t l, int32_t r0,
                                   int32_t c0) {
  const int total = p * q;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < parts; ++t) s += partial[(size_t)t * total + idx];
    C32[idx] = (float)s;
    if (Racc) {
      const int r = idx / q, c = idx - r * q;
      Racc[(size_t)(r0 + r) * l + c0 + c] += s;
    }
  }
}

// Y (rows x w, ld ldy) -= T (rows x w, ld ldt)
__global__ void subtract_kernel(float *__restrict__ Y, int64_t ldy, const float *__restrict__ T, int64_t ldt,
                                int64_t rows, int32_t w) {
  const int64_t total = rows * w;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / w;
    const int c = (int)(idx - r * w);
    Y[r * ldy + c] -= T[r * ldt + c];
  }
}

// Racc[r0 + r][r0 + c] = Rp[r][c] (w x w)
__global__ void place_block_kernel(const double *__restrict__ Rp, int32_t w, double *__restrict__ Racc, int32_t l,
                                   int32_t r0) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < w * w; idx += gridDim.x * blockDim.x) {
    const int r = idx / w, c = idx - r * w;
    Racc[(size_t)(r0 + r) * l + r0 + c] = Rp[idx];
  }
}

}  // namespace

size_t wide_orth_bytes(int64_t rows, int32_t l) {
  const int32_t m = (int32_t)ceil_div(l, kPanel);
  const int32_t parts = gram_ab_parts(rows);
  size_t off = 0;
  auto take = [&](size_t b) { off += (size_t)round_up((int64_t)b, 256); };
  take(sizeof(double) * (size_t)parts * kPanel * kPanel);                       // partials of one C_i
  take(sizeof(float) * (size_t)std::max(m - 1, 1) * kPanel * kPanel);           // C of each panel i < j
  take(sizeof(float) * (size_t)rows * kPanel);                                  // Q_i C
  take(sizeof(double) * (size_t)kPanel * kPanel);                               // a panel's R
  return off;
}

isvd_status wide_orth_enqueue(float *Q, int64_t ldq, int64_t rows, int32_t l, double *Racc, const OrthBufs &o,
                              char *wbuf, isvd_info *info, cudaStream_t s) {
  const int32_t m = (int32_t)ceil_div(l, kPanel);
  const int32_t parts = gram_ab_parts(rows);
  size_t off = 0;
  auto take = [&](size_t b) {
    char *p = wbuf + off;
    off += (size_t)round_up((int64_t)b, 256);
    return p;
  };
  double *partial = (double *)take(sizeof(double) * (size_t)parts * kPanel * kPanel);
  float *C32 = (float *)take(sizeof(float) * (size_t)std::max(m - 1, 1) * kPanel * kPanel);
  float *T = (float *)take(sizeof(float) * (size_t)rows * kPanel);
  double *Rp = (double *)take(sizeof(double) * (size_t)kPanel * kPanel);
  if (Racc) ISVD_CUDA_TRY(cudaMemsetAsync(Racc, 0, sizeof(double) * (size_t)l * l, s));
  for (int32_t j = 0; j < m; ++j) {
    float *Y = Q + (size_t)j * kPanel;
    const int32_t wj = std::min(kPanel, l - j * kPanel);
    for (int pass = 0; pass < 2 && j > 0; ++pass) {
      // every C_i from the same Y, then the subtractions (classical Gram-Schmidt)
      for (int32_t i = 0; i < j; ++i) {
        double *pi = partial;  // reduced before the next C_i is formed (stream order)
        bool tc = false;
        ISVD_CUDA_TRY(gram_ab_launch(Q + (size_t)i * kPanel, ldq, kPanel, Y, ldq, wj, rows, pi, parts, nullptr, &tc, s));
        if (!tc) ISVD_CUDA_TRY(tn_partial_launch(Q + (size_t)i * kPanel, ldq, Y, ldq, rows, kPanel, wj, pi, parts, s));
        wide_reduce_kernel<<<grid_for_elems((int64_t)kPanel * wj), 256, 0, s>>>(
            pi, parts, kPanel, wj, C32 + (size_t)i * kPanel * kPanel, Racc, l, i * kPanel, j * kPanel);
        ISVD_CUDA_TRY(cudaGetLastError());
      }
      for (int32_t i = 0; i < j; ++i) {
        // Y -= Q_i C_i: in the tensor-core epilogue, else through T
        bool launched = false;
        const float *Ci = C32 + (size_t)i * kPanel * kPanel;
        ISVD_CUDA_TRY(
            gemm_tc_launch(Q + (size_t)i * kPanel, ldq, rows, kPanel, Ci, wj, wj, Y, ldq, &launched, s, true));
        if (launched) continue;
        ISVD_CUDA_TRY(gemm_small_launch(Q + (size_t)i * kPanel, ldq, DT_F32, rows, kPanel, Ci, wj, wj, false, T,
                                        kPanel, DT_F32, PassGate{}, s));
        subtract_kernel<<<grid_for_elems(rows * wj), 256, 0, s>>>(Y, ldq, T, kPanel, rows, wj);
        ISVD_CUDA_TRY(cudaGetLastError());
      }
    }
    ISVD_TRY(orth_enqueue(Y, ldq, DT_F32, rows, wj, Racc ? Rp : nullptr, o, info, s));
    if (Racc) {
      place_block_kernel<<<grid_for_elems((int64_t)wj * wj), 256, 0, s>>>(Rp, wj, Racc, l, j * kPanel);
      ISVD_CUDA_TRY(cudaGetLastError());
    }
  }
  return ISVD_OK;
}

}  // namespace isvd
