// Sparse x tall-skinny dense product, nonzero-balanced form.
//
// Same row computation as spmm.cu (y_i = s r_i (sum_j a_ij w_j z_j + [self]
// w_i z_i) + a h_i x_i + sum_t alpha_t u_it c_t), organised for memory-level
// parallelism on power-law graphs:
//   - each warp takes a fixed chunk of CH consecutive nonzeros, whatever the
//     rows (hub rows are spread over many chunks, short rows share one);
//   - per batch of 32 nonzeros the warp loads the column indices, weights and
//     row numbers coalesced, then issues all the batch's gathers at once
//     (32 rows of 128 bytes of the column slab) into shared memory;
//   - a segmented sum over the batch (lane = column of the slab) accumulates
//     each row; rows that lie inside the chunk get their epilogue at once,
//     the first / last row of a chunk that crosses the chunk boundary is left
//     as a partial sum that a fix-up pass adds in chunk order
//     (deterministic).
// Column slabs are 128 bytes wide (32 FP32 or 64 BF16 columns) so that the
// gathered slab of the block is small enough to stay resident in L2.
#include "internal.h"

namespace isvd {
namespace {

constexpr int kWarps = 4;
constexpr int kThreads = kWarps * 32;

template <int DT>
struct CV;  // 16-byte vectors of the dense block, and the columns each lane owns in the scan

template <>
struct CV<DT_F32> {
  static constexpr int VN = 4, ES = 4, CPL = 1;  // CPL: columns per lane (slab = 32 * CPL)
  __device__ __forceinline__ static void unpack(uint4 x, float *v) {
    v[0] = __uint_as_float(x.x);
    v[1] = __uint_as_float(x.y);
    v[2] = __uint_as_float(x.z);
    v[3] = __uint_as_float(x.w);
  }
  __device__ __forceinline__ static float load1(const void *p) { return *reinterpret_cast<const float *>(p); }
  __device__ __forceinline__ static void store1(void *p, float v) { *reinterpret_cast<float *>(p) = v; }
};

template <>
struct CV<DT_BF16> {
  static constexpr int VN = 8, ES = 2, CPL = 2;
  __device__ __forceinline__ static void unpack(uint4 x, float *v) {
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&x);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __bfloat1622float2(h[k]);
      v[2 * k] = f.x;
      v[2 * k + 1] = f.y;
    }
  }
  __device__ __forceinline__ static float load1(const void *p) {
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(p));
  }
  __device__ __forceinline__ static void store1(void *p, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(p) = __float2bfloat16_rn(v);
  }
};

__device__ __forceinline__ uint64_t pol_keep() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t pol_stream() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
template <bool H>
__device__ __forceinline__ uint4 ldg16(const void *p, uint64_t pol) {
  uint4 v;
  if (H)
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
  else
    v = __ldg(reinterpret_cast<const uint4 *>(p));
  return v;
}
template <bool H>
__device__ __forceinline__ int32_t ldg_i(const int32_t *p, uint64_t pol) {
  int32_t v;
  if (H)
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  else
    v = __ldg(p);
  return v;
}

// Epilogue of one row for the columns this lane owns (col = lane + 32 c).
template <int DT>
__device__ __forceinline__ void row_epilogue(const SpmmArgs &a, const SpmmSlab &sl, int64_t r, const float *acc,
                                             int lane) {
  using V = CV<DT>;
  const float sc = a.scalar * (a.rowscale ? __ldg(a.rowscale + r) : 1.f);
  const float ws = a.self_term ? (a.colw ? __ldg(a.colw + r) : 1.f) : 0.f;
  const float as = sl.axpy ? a.ax_scalar * (a.ax_rowscale ? __ldg(a.ax_rowscale + r) : 1.f) : 0.f;
#pragma unroll
  for (int c = 0; c < V::CPL; ++c) {
    const int col = lane + 32 * c;
    if (col >= sl.width) continue;
    float v = acc[c];
    if (a.self_term) v = fmaf(ws, V::load1(reinterpret_cast<const char *>(sl.in) + ((size_t)r * sl.ldi + col) * V::ES), v);
    v *= sc;
    if (sl.axpy)
      v = fmaf(as, V::load1(reinterpret_cast<const char *>(sl.axpy) + ((size_t)r * sl.lda + col) * V::ES), v);
    for (int t = 0; t < a.lr_rank; ++t) {
      const int tu = t - a.lr_ones_first;
      const float u = (tu < 0 || !a.lr_u) ? 1.f : __ldg(a.lr_u + (size_t)r * a.lr_ldu + tu);
      v = fmaf(a.lr_alpha[t] * u, __ldg(a.lr_c + (size_t)t * a.lr_ldc + sl.col0 + col), v);
    }
    V::store1(reinterpret_cast<char *>(sl.out) + ((size_t)r * sl.ldo + col) * V::ES, v);
  }
}

template <int DT, bool H>
__global__ void __launch_bounds__(kThreads) spmm_chunk_kernel(const __grid_constant__ SpmmArgs a,
                                                              const int32_t *__restrict__ row_of, int64_t nnz,
                                                              int32_t CH, int64_t nchunks,
                                                              float *__restrict__ part, int64_t pw) {
  using V = CV<DT>;
  constexpr int SW = 32 * V::CPL;             // slab columns
  constexpr int G = SW / V::VN;               // lanes per gathered row (8 FP32, 8 BF16)
  constexpr int RPI = 32 / G;                 // gathered rows per warp instruction
  __shared__ __align__(16) float S[kWarps][32][SW + 4];  // 16-byte rows, bank-shifted
  __shared__ int32_t Js[kWarps][32];
  __shared__ float Ws[kWarps][32];
  __shared__ int32_t Rs[kWarps][32];
  const SpmmSlab &sl = a.slab[blockIdx.y];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int g = lane / G, gl = lane % G;
  const uint64_t pk = H ? pol_keep() : 0, ps = H ? pol_stream() : 0;
  const char *inb = reinterpret_cast<const char *>(sl.in) + (size_t)gl * V::VN * V::ES;
  const size_t ldb = (size_t)sl.ldi * V::ES;
  const bool active_g = gl * V::VN < sl.width;
  const int64_t nwarp = (int64_t)gridDim.x * kWarps;
  for (int64_t c = (int64_t)blockIdx.x * kWarps + wi; c < nchunks; c += nwarp) {
    const int64_t e0 = c * CH;
    const int64_t e1 = min(e0 + CH, nnz);
    // rows crossing the chunk boundaries
    const int32_t first_row = __ldg(row_of + e0), last_row = __ldg(row_of + e1 - 1);
    const int32_t head_row = (e0 > 0 && __ldg(row_of + e0 - 1) == first_row) ? first_row : -1;
    const int32_t tail_row = (e1 < nnz && __ldg(row_of + e1) == last_row) ? last_row : -1;
    float acc[V::CPL];
#pragma unroll
    for (int k = 0; k < V::CPL; ++k) acc[k] = 0.f;
    int32_t cur = first_row;
    auto flush = [&](int32_t row) {
      if (row == head_row || row == tail_row) {
        float *p = part + ((size_t)c * 2 + (row == head_row ? 0 : 1)) * pw + sl.col0;
#pragma unroll
        for (int k = 0; k < V::CPL; ++k)
          if (lane + 32 * k < sl.width) p[lane + 32 * k] = acc[k];
      } else {
        row_epilogue<DT>(a, sl, row, acc, lane);
      }
    };
    for (int64_t eb = e0; eb < e1; eb += 32) {
      const int nb = (int)((e1 - eb) < 32 ? (e1 - eb) : 32);
      {
        const int64_t e = eb + lane;
        int32_t j = 0, r = 0x7fffffff;
        float w = 0.f;
        if (lane < nb) {
          j = ldg_i<H>(a.colidx + e, ps);
          r = ldg_i<H>(row_of + e, ps);
          w = a.values ? __ldg(a.values + e) : 1.f;
          if (a.colw) w *= __ldg(a.colw + j);
        }
        Js[wi][lane] = j;
        Ws[wi][lane] = w;
        Rs[wi][lane] = r;
      }
      __syncwarp();
      // gathers: all of the batch's rows in flight at once
      uint4 raw[G];
#pragma unroll
      for (int t = 0; t < G; ++t) {
        const int q = t * RPI + g;
        raw[t] = (q < nb && active_g) ? ldg16<H>(inb + (size_t)Js[wi][q] * ldb, pk) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int t = 0; t < G; ++t) {
        const int q = t * RPI + g;
        float v[V::VN];
        V::unpack(raw[t], v);
        const float w = Ws[wi][q];
#pragma unroll
        for (int k = 0; k < V::VN; k += 4)
          *reinterpret_cast<float4 *>(&S[wi][q][gl * V::VN + k]) =
              make_float4(w * v[k], w * v[k + 1], w * v[k + 2], w * v[k + 3]);
      }
      __syncwarp();
      // segmented sum over the batch, lane = column
      for (int q = 0; q < nb; ++q) {
        const int32_t r = Rs[wi][q];
        if (r != cur) {
          flush(cur);
#pragma unroll
          for (int k = 0; k < V::CPL; ++k) acc[k] = 0.f;
          // rows without nonzeros between cur and r are handled by the empty-row pass
          cur = r;
        }
#pragma unroll
        for (int k = 0; k < V::CPL; ++k) acc[k] += S[wi][q][lane + 32 * k];
      }
      __syncwarp();
    }
    flush(cur);
  }
}

// Rows split across chunks: sum the tail partial of the first chunk and the
// head partials of the following chunks, in chunk order, then the epilogue.
template <int DT>
__global__ void __launch_bounds__(kThreads) spmm_chunk_fixup_kernel(const __grid_constant__ SpmmArgs a,
                                                                    const int4 *__restrict__ split, int32_t nsplit,
                                                                    const float *__restrict__ part, int64_t pw) {
  using V = CV<DT>;
  const SpmmSlab &sl = a.slab[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = (int64_t)gridDim.x * kWarps;
  for (int64_t i = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); i < nsplit; i += nwarp) {
    const int4 s = split[i];  // (row, first chunk, last chunk, 0)
    float acc[V::CPL];
#pragma unroll
    for (int k = 0; k < V::CPL; ++k) {
      const int col = lane + 32 * k;
      float v = 0.f;
      if (col < sl.width) {
        v = part[((size_t)s.y * 2 + 1) * pw + sl.col0 + col];
        for (int c = s.y + 1; c <= s.z; ++c) v += part[((size_t)c * 2) * pw + sl.col0 + col];
      }
      acc[k] = v;
    }
    row_epilogue<DT>(a, sl, s.x, acc, lane);
  }
}

// Rows with no nonzeros: the epilogue of an empty sum.
template <int DT>
__global__ void __launch_bounds__(kThreads) spmm_chunk_empty_kernel(const __grid_constant__ SpmmArgs a,
                                                                    const int32_t *__restrict__ rows, int32_t n) {
  using V = CV<DT>;
  const SpmmSlab &sl = a.slab[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = (int64_t)gridDim.x * kWarps;
  for (int64_t i = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); i < n; i += nwarp) {
    float acc[V::CPL];
#pragma unroll
    for (int k = 0; k < V::CPL; ++k) acc[k] = 0.f;
    row_epilogue<DT>(a, sl, rows[i], acc, lane);
  }
}

template <int DT, bool H>
cudaError_t launch(const SpmmArgs &a, const ChunkPlan &cp, float *part, int64_t pw, cudaStream_t s) {
  const int64_t cap = (int64_t)kNumSMs * 8;
  if (cp.nchunks > 0) {
    int64_t bx = ceil_div(cp.nchunks, kWarps);
    if (bx > cap) bx = cap;
    spmm_chunk_kernel<DT, H><<<dim3((unsigned)bx, (unsigned)a.nslabs), kThreads, 0, s>>>(
        a, cp.row_of, cp.nnz, cp.CH, cp.nchunks, part, pw);
  }
  if (cp.nsplit > 0) {
    int64_t bx = ceil_div(cp.nsplit, kWarps);
    if (bx > cap) bx = cap;
    spmm_chunk_fixup_kernel<DT><<<dim3((unsigned)bx, (unsigned)a.nslabs), kThreads, 0, s>>>(a, cp.split, cp.nsplit,
                                                                                         part, pw);
  }
  if (cp.nempty > 0) {
    int64_t bx = ceil_div(cp.nempty, kWarps);
    if (bx > cap) bx = cap;
    spmm_chunk_empty_kernel<DT><<<dim3((unsigned)bx, (unsigned)a.nslabs), kThreads, 0, s>>>(a, cp.empty, cp.nempty);
  }
  return cudaGetLastError();
}

}  // namespace

int chunk_slab_cols(int dtype) { return dtype == DT_F32 ? 32 : 64; }

cudaError_t spmm_chunk_launch(const SpmmArgs &a, int dtype, const ChunkPlan &cp, float *part, int64_t pw,
                              cudaStream_t s) {
  if (a.rows == 0 || a.nslabs == 0) return cudaSuccess;
  if (a.cache_hints)
    return dtype == DT_F32 ? launch<DT_F32, true>(a, cp, part, pw, s) : launch<DT_BF16, true>(a, cp, part, pw, s);
  return dtype == DT_F32 ? launch<DT_F32, false>(a, cp, part, pw, s) : launch<DT_BF16, false>(a, cp, part, pw, s);
}

}  // namespace isvd
