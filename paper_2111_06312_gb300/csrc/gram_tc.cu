// Gram matrix W = Q^T Q of a tall block on the 5th-generation tensor cores
// (tcgen05), the contraction of CholeskyQR (Alg. 2: L = chol(Q^T Q)).
//
// Q is n x l row-major (l <= 160).  Each CTA reduces a contiguous range of
// rows: 32 (FP32) or 64 (BF16) rows at a time are copied raw into shared
// memory with cp.async (four chunks in flight), then producer warps write the
// transposed chunk as a K-major operand tile (128-byte swizzle): row m of the
// tile holds column m of Q over the chunk's rows.  The same tile is both MMA
// operands (A rows and B rows are both columns of Q):
//   tile 1: W[0:128, 0:N1]      M = 128, N = round16(l)
//   tile 2: W[128:256, 128:N1]  M = 128, N = round16(l - 128)   (l > 128)
// and W[128:, :128] is the transpose of tile 1's right part.  FP32 blocks use
// 3xTF32 (x = hi + lo with hi in TF32: hi*hi + hi*lo + lo*hi); BF16 blocks use
// one BF16 MMA (exact products).  Accumulators stay in tensor memory for the
// whole row range; each CTA writes its l x l partial, combined in FP64 in a
// fixed order by gram_reduce (deterministic).
#include <mutex>

#include "internal.h"
#include "tc_common.cuh"

namespace isvd {
namespace {

using namespace tc;

constexpr int kProdWarps = 8;
constexpr int kProd = kProdWarps * 32;
constexpr int kThreads = kProd + 32;  // + MMA warp
constexpr int kRawStages = 4;
constexpr int kTileStages = 2;
constexpr int kTmemCols = 256;
constexpr int kTile2Col = 192;

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void producer_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kProd) : "memory"); }

template <int DT>
struct GramCfg {
  static constexpr bool F32 = DT == DT_F32;
  static constexpr int ES = F32 ? 4 : 2;
  static constexpr int BK = F32 ? 32 : 64;  // rows per chunk = 128 bytes of K per tile row
  static constexpr int NT = F32 ? 2 : 1;    // tiles per stage (hi, lo)
};

template <int DT>
__global__ void __launch_bounds__(kThreads, 1)
    gram_tc_kernel(const void *__restrict__ Qv, int64_t ldq, int64_t rows, int32_t l, float *__restrict__ partial,
                   int64_t rows_per_cta, const int32_t *gate_state, int32_t gate_pass, int32_t *err_state) {
  using C = GramCfg<DT>;
  if (gate_state && gate_pass > 2 && gate_state[0] + 2 < gate_pass) return;
  const int MT = l > 128 ? 256 : 128;
  const int tile_bytes = MT * 128;
  const int lp = (l + 7) & ~7;                     // raw row pitch in elements (16-byte multiple)
  const int raw_bytes = C::BK * lp * C::ES;
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t full[kTileStages], empty[kTileStages], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  unsigned char *sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
  unsigned char *tiles = sm;                                       // [kTileStages][NT][tile]
  unsigned char *raw = sm + (size_t)kTileStages * C::NT * tile_bytes;  // [kRawStages][raw]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = min(rows, r0 + rows_per_cta);
  const int nchunks = r1 > r0 ? (int)((r1 - r0 + C::BK - 1) / C::BK) : 0;
  const int N1 = (l + 15) & ~15;
  const int N2 = l > 128 ? ((l - 128 + 15) & ~15) : 0;

  for (int i = tid; i < kTileStages * C::NT * tile_bytes / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(tiles)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int s = 0; s < kTileStages; ++s) {
      mbar_init(&full[s], kProd);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  fence_async_shared();
  __syncthreads();
  if (warp == 0) tmem_alloc(&tmem_slot, kTmemCols);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp < kProdWarps) {
    // ---------------- producers ----------------
    const char *Q = reinterpret_cast<const char *>(Qv);
    const int pieces = (l * C::ES + 15) / 16;  // 16-byte pieces per row
    auto issue = [&](int c) {
      if (c < nchunks) {
        unsigned char *rb = raw + (size_t)(c % kRawStages) * raw_bytes;
        const int64_t row0 = r0 + (int64_t)c * C::BK;
        for (int t = tid; t < C::BK * pieces; t += kProd) {
          const int rr = t / pieces, pc = t - rr * pieces;
          const int64_t r = row0 + rr;
          if (r < r1) cp_async16(smem_u32(rb + (size_t)rr * lp * C::ES + pc * 16), Q + ((size_t)r * ldq) * C::ES + pc * 16);
        }
      }
      cp_async_commit();
    };
    for (int c = 0; c < kRawStages - 1; ++c) issue(c);
    for (int c = 0; c < nchunks; ++c) {
      issue(c + kRawStages - 1);
      cp_async_wait<kRawStages - 1>();
      const int s = c % kTileStages;
      // one thread waits for the tile stage to be free; the decision is shared
      if (tid == 0 && c >= kTileStages && !mbar_wait(&empty[s], ((c / kTileStages) & 1) ^ 1)) {
        abort_flag = 1;
        if (err_state) atomicExch(&err_state[2], 1);
      }
      producer_bar();  // chunk c is in shared memory for every producer; stage s is free
      if (abort_flag) break;
      const unsigned char *rb = raw + (size_t)(c % kRawStages) * raw_bytes;
      const int64_t row0 = r0 + (int64_t)c * C::BK;
      const int valid = (int)((r1 - row0) < C::BK ? (r1 - row0) : C::BK);
      unsigned char *thi = tiles + (size_t)(s * C::NT) * tile_bytes;
      // task (m, kq): column m of Q over 16 bytes of K (4 FP32 or 8 BF16 rows)
      for (int t = tid; t < l * 8; t += kProd) {
        const int m = t % l, kq = t / l;
        if (C::F32) {
          float hi[4], lo[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int rr = 4 * kq + j;
            const float x = rr < valid ? reinterpret_cast<const float *>(rb + (size_t)rr * lp * 4)[m] : 0.f;
            split_tf32(x, hi[j], lo[j]);
          }
          *reinterpret_cast<float4 *>(thi + sw128(m, 16 * kq)) = make_float4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<float4 *>(thi + tile_bytes + sw128(m, 16 * kq)) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        } else {
          unsigned short v[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int rr = 8 * kq + j;
            v[j] = rr < valid ? reinterpret_cast<const unsigned short *>(rb + (size_t)rr * lp * 2)[m] : (unsigned short)0;
          }
          uint4 w;
          w.x = v[0] | ((uint32_t)v[1] << 16);
          w.y = v[2] | ((uint32_t)v[3] << 16);
          w.z = v[4] | ((uint32_t)v[5] << 16);
          w.w = v[6] | ((uint32_t)v[7] << 16);
          *reinterpret_cast<uint4 *>(thi + sw128(m, 16 * kq)) = w;
        }
      }
      fence_async_shared();
      mbar_arrive(&full[s]);
      producer_bar();  // raw buffer of chunk c may be refilled after this
    }
    cp_async_wait<0>();
  } else if (lane == 0) {
    // ---------------- MMA issuer ----------------
    const uint32_t fmt = C::F32 ? 2u : 1u;
    const uint32_t id1 = idesc(fmt, 128, N1);
    const uint32_t id2 = idesc(fmt, 128, N2 > 0 ? N2 : 16);
    for (int c = 0; c < nchunks; ++c) {
      const int s = c % kTileStages;
      if (abort_flag || !mbar_wait(&full[s], (c / kTileStages) & 1)) {
        if (err_state) atomicExch(&err_state[2], 1);
        break;
      }
      fence_after();
      const uint32_t hi = smem_u32(tiles + (size_t)(s * C::NT) * tile_bytes);
      const uint32_t lo = hi + tile_bytes;
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
        const uint64_t ah = desc_sw128(hi + kk * 32, 1024);
        if (C::F32) {
          const uint64_t al = desc_sw128(lo + kk * 32, 1024);
          mma_tf32(tmem, ah, ah, id1, acc);
          mma_tf32(tmem, ah, al, id1, 1u);
          mma_tf32(tmem, al, ah, id1, 1u);
          if (N2) {
            const uint64_t bh = desc_sw128(hi + 16384 + kk * 32, 1024);
            const uint64_t bl = desc_sw128(lo + 16384 + kk * 32, 1024);
            mma_tf32(tmem + kTile2Col, bh, bh, id2, acc);
            mma_tf32(tmem + kTile2Col, bh, bl, id2, 1u);
            mma_tf32(tmem + kTile2Col, bl, bh, id2, 1u);
          }
        } else {
          mma_bf16(tmem, ah, ah, id1, acc);
          if (N2) {
            const uint64_t bh = desc_sw128(hi + 16384 + kk * 32, 1024);
            mma_bf16(tmem + kTile2Col, bh, bh, id2, acc);
          }
        }
      }
      commit(&empty[s]);
    }
    commit(&done);
  }
  // ---------------- epilogue: TMEM -> partial ----------------
  __syncwarp();
  const bool ok = mbar_wait(&done, 0);
  if (!ok && err_state && tid == 0) atomicExch(&err_state[2], 1);
  fence_after();
  float *P = partial + (size_t)blockIdx.x * l * l;
  if (nchunks == 0 || !ok) {
    for (int i = tid; i < l * l; i += blockDim.x) P[i] = 0.f;
  } else if (warp < 4) {
    const int i = warp * 32 + lane;  // W row
    uint32_t r[32];
    for (int cb = 0; cb < N1; cb += 32) {
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + cb, r);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = cb + j;
        if (i < l && n < l) {
          const float v = __uint_as_float(r[j]);
          P[(size_t)i * l + n] = v;
          if (n >= 128) P[(size_t)n * l + i] = v;  // W[128:, :128] by symmetry
        }
      }
    }
  } else if (warp < 8 && N2 > 0) {
    const int w4 = warp - 4;
    const int i = 128 + w4 * 32 + lane;
    uint32_t r[32];
    for (int cb = 0; cb < N2; cb += 32) {
      tmem_ld32(tmem + ((uint32_t)(w4 * 32) << 16) + kTile2Col + cb, r);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = 128 + cb + j;
        if (i < l && n < l) P[(size_t)i * l + n] = __uint_as_float(r[j]);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

__global__ void gram_reduce_tc_kernel(const float *partial, int32_t n_part, int32_t l, double *W,
                                      const int32_t *gate_state, int32_t gate_pass) {
  if (gate_state && gate_pass > 2 && gate_state[0] + 2 < gate_pass) return;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)l * l) return;
  double s = 0.0;
  for (int p = 0; p < n_part; ++p) s += (double)partial[(int64_t)p * l * l + idx];
  W[idx] = s;
}

template <int DT>
size_t gram_tc_smem(int32_t l) {
  using C = GramCfg<DT>;
  const int MT = l > 128 ? 256 : 128;
  const int lp = (l + 7) & ~7;
  return (size_t)kTileStages * C::NT * MT * 128 + (size_t)kRawStages * C::BK * lp * C::ES + 1024;
}

std::once_flag g_once;
cudaError_t g_err = cudaSuccess;

}  // namespace

cudaError_t gram_tc_init() {
  std::call_once(g_once, [] {
    cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel<DT_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gram_tc_smem<DT_F32>(ISVD_MAX_BLOCK));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gram_tc_kernel<DT_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)gram_tc_smem<DT_BF16>(ISVD_MAX_BLOCK));
    g_err = e;
  });
  return g_err;
}

int32_t gram_partials(int64_t rows) {
  int64_t p = ceil_div(rows, 64);
  if (p > kNumSMs) p = kNumSMs;
  if (p < 1) p = 1;
  return (int32_t)p;
}

cudaError_t gram_launch(const void *Q, int64_t ldq, int dtype, int64_t rows, int32_t l, float *partial, int32_t n_part,
                        double *W, PassGate g, cudaStream_t s) {
  cudaError_t e = gram_tc_init();
  if (e != cudaSuccess) return e;
  const int bk = dtype == DT_F32 ? 32 : 64;
  const int64_t rpc = round_up(ceil_div(rows, n_part), bk);
  const int32_t used = (int32_t)std::max<int64_t>(1, ceil_div(rows, rpc));
  int32_t *err = const_cast<int32_t *>(g.state);
  if (dtype == DT_F32)
    gram_tc_kernel<DT_F32><<<used, kThreads, gram_tc_smem<DT_F32>(l), s>>>(Q, ldq, rows, l, partial, rpc, g.state,
                                                                            g.pass, err);
  else
    gram_tc_kernel<DT_BF16><<<used, kThreads, gram_tc_smem<DT_BF16>(l), s>>>(Q, ldq, rows, l, partial, rpc, g.state,
                                                                              g.pass, err);
  gram_reduce_tc_kernel<<<(unsigned)ceil_div((int64_t)l * l, 256), 256, 0, s>>>(partial, used, l, W, g.state, g.pass);
  return cudaGetLastError();
}

}  // namespace isvd
