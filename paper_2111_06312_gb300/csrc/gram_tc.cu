// Gram matrix W = Q^T Q of a tall block on the 5th-generation tensor cores
// (tcgen05), the contraction of CholeskyQR (Alg. 2: L = chol(Q^T Q)).
//
// Q is n x l row-major (l <= 160).  Each CTA reduces a contiguous range of
// rows: 32 (FP32) or 64 (BF16) rows at a time are copied raw into a ring of
// shared-memory stages (one bulk copy per chunk when the rows are contiguous,
// else 16-byte cp.async pieces; as many stages as the shared memory holds),
// then producer warps write the transposed chunk as a K-major operand tile
// (128-byte swizzle; three tile stages): row m of the tile holds column m of
// Q over the chunk's rows.  The same tile is both MMA
// operands (A rows and B rows are both columns of Q):
//   tile 1: W[0:128, 0:N1]      M = 128, N = round16(l)
//   tile 2: W[128:256, 128:N1]  M = 128, N = round16(l - 128)   (l > 128)
// and W[128:, :128] is the transpose of tile 1's right part.  FP32 blocks use
// 3xTF32 (x = hi + lo with hi in TF32: hi*hi + hi*lo + lo*hi); BF16 blocks use
// one BF16 MMA (exact products).  The tensor cores' FP32 accumulation loses
// a little on every addition, and over thousands of rows the loss adds up
// (CholeskyQR2's orthogonality fell linearly with the rows per CTA, 1.2e-4
// at 6,600), so each 384-row segment is accumulated in tensor memory (two
// buffers, alternating) and eight epilogue warps add it, with round-to-nearest
// FP32 additions, into the CTA's partial held in their registers (thread =
// one row of W and half of its columns) while the next segment is multiplied.
// The segment sums are few (17 per CTA at 10^6 rows), so this adds only
// ~sqrt(17) u of relative error; the partials are written once at the end and
// combined in FP64 in a fixed order by gram_reduce (deterministic).
#include <mutex>

#include "internal.h"
#include "tc_common.cuh"

namespace isvd {
namespace {

using namespace tc;

constexpr int kProdWarps = 7;  // with the MMA warp and 8 epilogue warps: 16 warps, 128 registers each
constexpr int kProd = kProdWarps * 32;
constexpr int kMmaWarp = kProdWarps;       // warp 7
constexpr int kEpiWarp0 = kProdWarps + 1;  // warps 8..15: epilogue (two per TMEM lane quarter)
constexpr int kEpiThreads = 256;
constexpr int kThreads = kProd + 32 + kEpiThreads;
constexpr int kHalfBlocks = 5;  // 16-column blocks of tile 1 per epilogue half (N1 <= 160)
constexpr int kMaxRaw = 8;              // raw chunk stages at most
constexpr int kMaxSmem = 221 * 1024;    // dynamic shared memory; the static part (tile-2 partial, barriers) takes the rest
constexpr int kTileStages = 3;
constexpr int kTmemCols = 512;
constexpr int kAccCols = 256;  // accumulator buffer b at column b * kAccCols
constexpr int kTile2Col = 192;
constexpr int kSegRows = 384;  // rows summed in tensor memory before promotion to FP64

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
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

// raw stages that fit beside the tile stages (kMaxRaw at most, 2 at least)
template <int DT>
__host__ __device__ inline int gram_raw_stages(int32_t l) {
  using C = GramCfg<DT>;
  const int TR = l > 128 ? (l + 7) & ~7 : 128;
  const int lp = (l + 7) & ~7;
  const long tiles = (long)kTileStages * C::NT * TR * 128;
  const long raw = (long)C::BK * lp * C::ES;
  long r = (kMaxSmem - 1024 - tiles) / raw;
  return (int)(r > kMaxRaw ? kMaxRaw : (r < 2 ? 2 : r));
}

template <int DT>
__global__ void __launch_bounds__(kThreads, 1)
    gram_tc_kernel(const void *__restrict__ Qv, int64_t ldq, int64_t rows, int32_t l, float *__restrict__ partial,
                   int64_t rows_per_cta, int32_t bulk, const int32_t *gate_state, int32_t gate_pass,
                   int32_t *err_state) {
  using C = GramCfg<DT>;
  if (gate_state && gate_pass > 2 && gate_state[0] + 2 < gate_pass) return;
  // A tile holds round8(l) rows (at least 128, the MMA's M).  For l > 128 the
  // second MMA (M = 128 from row 128) also reads the bytes after the tile's
  // last row: they lie inside the next buffer of the same allocation and only
  // reach accumulator rows >= l - 128 of that MMA, which are never read.
  const int TR = l > 128 ? (l + 7) & ~7 : 128;
  const int tile_bytes = TR * 128;
  const int lp = (l + 7) & ~7;                     // raw row pitch in elements (16-byte multiple)
  const int raw_bytes = C::BK * lp * C::ES;
  const int R = gram_raw_stages<DT>(l);
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t full[kTileStages], empty[kTileStages], seg_full[2], seg_free[2], raw_full[kMaxRaw];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  unsigned char *sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
  unsigned char *tiles = sm;                                       // [kTileStages][NT][tile]
  unsigned char *raw = sm + (size_t)kTileStages * C::NT * tile_bytes;  // [R][raw]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = min(rows, r0 + rows_per_cta);
  const int nchunks = r1 > r0 ? (int)((r1 - r0 + C::BK - 1) / C::BK) : 0;
  constexpr int F = kSegRows / C::BK;  // chunks per segment
  const int nseg = (nchunks + F - 1) / F;
  const int N1 = (l + 15) & ~15;
  const int N2 = l > 128 ? ((l - 128 + 15) & ~15) : 0;

  for (int i = tid; i < kTileStages * C::NT * tile_bytes / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(tiles)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int s = 0; s < kTileStages; ++s) {
      mbar_init(&full[s], 1);  // one arrive after the producers' barrier
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&seg_full[b], 1);
      mbar_init(&seg_free[b], kEpiThreads);
    }
    // a raw stage completes on the bulk copy's bytes, or on every producer's cp.async pieces
    for (int s = 0; s < R; ++s) mbar_init(&raw_full[s], bulk ? 1 : kProd);
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
    int issued = 0;
    auto issue = [&](int c) {
      if (c >= nchunks) return;
      unsigned char *rb = raw + (size_t)(c % R) * raw_bytes;
      const int64_t row0 = r0 + (int64_t)c * C::BK;
      const int valid = (int)((r1 - row0) < C::BK ? (r1 - row0) : C::BK);
      if (bulk) {
        // rows row0.. are contiguous (ldq == lp): one copy of valid * lp elements
        if (tid == 0) {
          const uint32_t bytes = (uint32_t)valid * lp * C::ES;
          mbar_expect_tx(&raw_full[c % R], bytes);
          bulk_g2s(smem_u32(rb), Q + (size_t)row0 * ldq * C::ES, bytes, &raw_full[c % R]);
        }
      } else {
        int rr = tid / pieces, pc = tid - rr * pieces;
        const int drr = kProd / pieces, dpc = kProd - drr * pieces;
        while (rr < valid) {
          cp_async16(smem_u32(rb + (size_t)rr * lp * C::ES + pc * 16), Q + ((size_t)(row0 + rr) * ldq) * C::ES + pc * 16);
          rr += drr;
          pc += dpc;
          if (pc >= pieces) {
            pc -= pieces;
            ++rr;
          }
        }
        cp_async_arrive_noinc(&raw_full[c % R]);
      }
      issued = c + 1;
    };
    // task (m, kq) of the transform: column m of Q over 16 bytes of K (4 FP32
    // or 8 BF16 rows).  This thread's tasks (m0 + i kProd) are the same for
    // every chunk: their shared-memory offsets are computed once (source: the
    // task's first raw row; destination: the swizzled tile position).
    constexpr int kMaxTasks = (ISVD_MAX_BLOCK * 8 + kProd - 1) / kProd;
    const int rs = lp * C::ES;  // raw row pitch in bytes
    uint32_t src_off[kMaxTasks], dst_off[kMaxTasks];
    int row_of[kMaxTasks];
    int ntask = 0;
#pragma unroll
    for (int i = 0; i < kMaxTasks; ++i) {
      const int t = tid + i * kProd;
      const int m = t % l, kq = t / l;
      row_of[i] = (C::F32 ? 4 : 8) * kq;
      src_off[i] = (uint32_t)(row_of[i] * rs + m * C::ES);
      dst_off[i] = sw128(m, 16 * kq);
      if (t < l * 8) ntask = i + 1;
    }
    int c = 0;
    for (int j = 0; j < R - 1; ++j) issue(j);
    for (; c < nchunks; ++c) {
      issue(c + R - 1);  // into the raw stage transformed in the previous iteration
      const int s = c % kTileStages;
      bool ok = mbar_wait(&raw_full[c % R], (uint32_t)((c / R) & 1));
      // one thread waits for the tile stage to be free; the decision is shared
      if (tid == 0 && c >= kTileStages && !mbar_wait(&empty[s], ((c / kTileStages) & 1) ^ 1)) ok = false;
      if (!ok) {
        abort_flag = 1;
        if (err_state) atomicExch(&err_state[2], 1);
      }
      producer_bar();  // chunk c is in shared memory; stage s is free
      if (abort_flag) break;
      const unsigned char *rb = raw + (size_t)(c % R) * raw_bytes;
      const int64_t row0 = r0 + (int64_t)c * C::BK;
      const int valid = (int)((r1 - row0) < C::BK ? (r1 - row0) : C::BK);
      unsigned char *thi = tiles + (size_t)(s * C::NT) * tile_bytes;
#pragma unroll
      for (int i = 0; i < kMaxTasks; ++i) {
        if (i >= ntask) break;
        const unsigned char *src = rb + src_off[i];
        const int rr0 = row_of[i];  // first raw row of the task (rows past valid read as 0)
        if (C::F32) {
          float hi[4], lo[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const float x = (valid == C::BK || rr0 + j < valid) ? *reinterpret_cast<const float *>(src + j * rs) : 0.f;
            split_tf32(x, hi[j], lo[j]);
          }
          *reinterpret_cast<float4 *>(thi + dst_off[i]) = make_float4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<float4 *>(thi + tile_bytes + dst_off[i]) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        } else {
          uint32_t v[8];
#pragma unroll
          for (int j = 0; j < 8; ++j)
            v[j] = (valid == C::BK || rr0 + j < valid) ? *reinterpret_cast<const unsigned short *>(src + j * rs) : 0u;
          *reinterpret_cast<uint4 *>(thi + dst_off[i]) =
              make_uint4(v[0] | (v[1] << 16), v[2] | (v[3] << 16), v[4] | (v[5] << 16), v[6] | (v[7] << 16));
        }
      }
      fence_async_shared();
      producer_bar();  // the tile is written (and the raw stage of chunk c may be refilled)
      if (tid == 0) mbar_arrive(&full[s]);
    }
    // after an abort, let the copies already issued land before the CTA exits
    for (int j = c; j < issued; ++j) mbar_wait(&raw_full[j % R], (uint32_t)((j / R) & 1));
    cp_async_wait<0>();
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t fmt = C::F32 ? 2u : 1u;
      const uint32_t id1 = idesc(fmt, 128, N1);
      const uint32_t id2 = idesc(fmt, 128, N2 > 0 ? N2 : 16);
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % kTileStages;
        const int seg = c / F, b = seg & 1, cs = c - seg * F;
        if (cs == 0 && seg >= 2 && !mbar_wait(&seg_free[b], (uint32_t)(((seg >> 1) - 1) & 1))) {
          if (err_state) atomicExch(&err_state[2], 1);
          abort_flag = 1;
          break;
        }
        if (abort_flag || !mbar_wait(&full[s], (c / kTileStages) & 1)) {
          if (err_state) atomicExch(&err_state[2], 1);
          abort_flag = 1;
          break;
        }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(b * kAccCols);
        const uint32_t hi = smem_u32(tiles + (size_t)(s * C::NT) * tile_bytes);
        const uint32_t lo = hi + tile_bytes;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t acc = (cs > 0 || kk > 0) ? 1u : 0u;
          const uint64_t ah = desc_sw128(hi + kk * 32, 1024);
          if (C::F32) {
            const uint64_t al = desc_sw128(lo + kk * 32, 1024);
            mma_tf32(d, ah, ah, id1, acc);
            mma_tf32(d, ah, al, id1, 1u);
            mma_tf32(d, al, ah, id1, 1u);
            if (N2) {
              const uint64_t bh = desc_sw128(hi + 16384 + kk * 32, 1024);
              const uint64_t bl = desc_sw128(lo + 16384 + kk * 32, 1024);
              mma_tf32(d + kTile2Col, bh, bh, id2, acc);
              mma_tf32(d + kTile2Col, bh, bl, id2, 1u);
              mma_tf32(d + kTile2Col, bl, bh, id2, 1u);
            }
          } else {
            mma_bf16(d, ah, ah, id1, acc);
            if (N2) {
              const uint64_t bh = desc_sw128(hi + 16384 + kk * 32, 1024);
              mma_bf16(d + kTile2Col, bh, bh, id2, acc);
            }
          }
        }
        commit(&empty[s]);
        if (cs == F - 1 || c == nchunks - 1) commit(&seg_full[b]);
      }
    }
  } else {
    // ---------------- epilogue: each segment's sums -> the register partial ----------------
    // Partial layout: P[n][i] = W[i][n] for i < 128 (tile 1, every n < l) and
    // P[128 + b][128 + a] = W[128 + a][128 + b] (tile 2); W is symmetric and the
    // reduction maps the rest.  Thread (quarter q, half h, lane) owns W row
    // i = 32 q + lane, columns [80 h, 80 h + 80) of tile 1; the quarter-0 warp
    // of half 1 also owns tile 2's rows (partial in shared memory).
    __shared__ float t2part[32 * 32];  // [column][lane]
    const int q = warp & 3;  // a warp reads the tensor-memory lanes of its quarter, 32 (warp % 4)
    const int h = (warp - kEpiWarp0) >> 2;
    const int i = q * 32 + lane;
    const int nblk = N1 / 16;
    const bool owns_t2 = N2 > 0 && q == 0 && h == 1;
    float part[kHalfBlocks][16];
#pragma unroll
    for (int k = 0; k < kHalfBlocks; ++k)
#pragma unroll
      for (int j = 0; j < 16; ++j) part[k][j] = 0.f;
    if (owns_t2)
      for (int c = 0; c < 32; ++c) t2part[c * 32 + lane] = 0.f;
    uint32_t v[16];
    for (int seg = 0; seg < nseg; ++seg) {
      const int b = seg & 1;
      if (!mbar_wait(&seg_full[b], (uint32_t)((seg >> 1) & 1))) {
        if (err_state && lane == 0) atomicExch(&err_state[2], 1);
        break;
      }
      fence_after();
      const uint32_t d = tmem + (uint32_t)(b * kAccCols) + ((uint32_t)(q * 32) << 16);
#pragma unroll
      for (int k = 0; k < kHalfBlocks; ++k) {
        const int blk = h * kHalfBlocks + k;
        if (blk < nblk) {
          tmem_ld16(d + (uint32_t)(blk * 16), v);
#pragma unroll
          for (int j = 0; j < 16; ++j) part[k][j] = __fadd_rn(part[k][j], __uint_as_float(v[j]));
        }
      }
      if (owns_t2)
        for (int c0 = 0; c0 < N2; c0 += 16) {
          tmem_ld16(d + (uint32_t)(kTile2Col + c0), v);
#pragma unroll
          for (int j = 0; j < 16; ++j)
            t2part[(c0 + j) * 32 + lane] = __fadd_rn(t2part[(c0 + j) * 32 + lane], __uint_as_float(v[j]));
        }
      fence_before();
      mbar_arrive(&seg_free[b]);
    }
    // one write of the partial (zero when this CTA had no rows)
    float *P = partial + (size_t)blockIdx.x * l * l;
    if (i < l) {
#pragma unroll
      for (int k = 0; k < kHalfBlocks; ++k) {
        const int c0 = (h * kHalfBlocks + k) * 16;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < l) P[(size_t)(c0 + j) * l + i] = part[k][j];
      }
    }
    if (owns_t2 && 128 + lane < l)
      for (int c = 0; c < l - 128; ++c) P[(size_t)(128 + c) * l + 128 + lane] = t2part[c * 32 + lane];
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// W[r][c] = sum over partials of P[r][c] (in FP64), except the block
// r < 128 <= c, which tile 1 stored transposed (P[c][r]).  A block covers
// kRedCols elements with kRedGroups thread rows; row g sums partials g,
// g + kRedGroups, ... (eight interleaved sums per thread, so that loads
// overlap), and the group sums are added in a fixed order (deterministic).
constexpr int kRedCols = 64, kRedGroups = 4;

__global__ void __launch_bounds__(kRedCols *kRedGroups)
    gram_reduce_tc_kernel(const float *partial, int32_t n_part, int32_t l, double *W, const int32_t *gate_state,
                          int32_t gate_pass) {
  if (gate_state && gate_pass > 2 && gate_state[0] + 2 < gate_pass) return;
  __shared__ double part[kRedGroups][kRedCols];
  const int g = threadIdx.y;
  const int64_t idx = (int64_t)blockIdx.x * kRedCols + threadIdx.x;
  double total = 0.0;
  if (idx < (int64_t)l * l) {
    const int r = (int)(idx / l), c = (int)(idx - (int64_t)r * l);
    const int64_t src = (r < 128 && c >= 128) ? (int64_t)c * l + r : idx;
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const int64_t stride = (int64_t)l * l;
    int p = g;
    for (; p + 7 * kRedGroups < n_part; p += 8 * kRedGroups)
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] += (double)partial[(int64_t)(p + u * kRedGroups) * stride + src];
#pragma unroll
    for (int u = 0; u < 7; ++u)
      if (p + u * kRedGroups < n_part) acc[u] += (double)partial[(int64_t)(p + u * kRedGroups) * stride + src];
    total = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  }
  part[g][threadIdx.x] = total;
  __syncthreads();
  if (g == 0 && idx < (int64_t)l * l) {
    double w = part[0][threadIdx.x];
#pragma unroll
    for (int t = 1; t < kRedGroups; ++t) w += part[t][threadIdx.x];
    W[idx] = w;
  }
}

template <int DT>
size_t gram_tc_smem(int32_t l) {
  using C = GramCfg<DT>;
  const int TR = l > 128 ? (l + 7) & ~7 : 128;
  const int lp = (l + 7) & ~7;
  // tiles, then the raw ring (at least 16 KB after the last tile, see above)
  return (size_t)kTileStages * C::NT * TR * 128 + (size_t)gram_raw_stages<DT>(l) * C::BK * lp * C::ES + 1024;
}

std::once_flag g_once;
cudaError_t g_err = cudaSuccess;

}  // namespace

cudaError_t gram_tc_init() {
  std::call_once(g_once, [] {
    cudaError_t e = cudaFuncSetAttribute(gram_tc_kernel<DT_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(gram_tc_kernel<DT_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
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

cudaError_t gram_launch(const void *Q, int64_t ldq, int dtype, int64_t rows, int32_t l, double *partial, int32_t n_part,
                        double *W, PassGate g, cudaStream_t s) {
  cudaError_t e = gram_tc_init();
  if (e != cudaSuccess) return e;
  const int bk = dtype == DT_F32 ? 32 : 64;
  const int64_t rpc = round_up(ceil_div(rows, n_part), bk);
  const int32_t used = (int32_t)std::max<int64_t>(1, ceil_div(rows, rpc));
  int32_t *err = const_cast<int32_t *>(g.state);
  // one bulk copy per chunk when consecutive rows are contiguous (pitch = the
  // 16-byte-rounded row) and the block starts on a 16-byte boundary
  const int32_t bulk = ldq == ((l + 7) & ~7) && ((uintptr_t)Q & 15) == 0;
  float *P = reinterpret_cast<float *>(partial);  // FP32 partials in the FP64-sized buffer
  if (dtype == DT_F32)
    gram_tc_kernel<DT_F32><<<used, kThreads, gram_tc_smem<DT_F32>(l), s>>>(Q, ldq, rows, l, P, rpc, bulk, g.state,
                                                                            g.pass, err);
  else
    gram_tc_kernel<DT_BF16><<<used, kThreads, gram_tc_smem<DT_BF16>(l), s>>>(Q, ldq, rows, l, P, rpc, bulk, g.state,
                                                                              g.pass, err);
  gram_reduce_tc_kernel<<<(unsigned)ceil_div((int64_t)l * l, kRedCols), dim3(kRedCols, kRedGroups), 0, s>>>(
      P, used, l, W, g.state, g.pass);
  return cudaGetLastError();
}

}  // namespace isvd
