// C = A^T B over a long row dimension on the 5th-generation tensor cores
// (tcgen05): the weight gradient dW = X^T [dY | N dY | N^2 dY] of the linear
// model on M = [X | N X | N^2 X] (Sec. 3.3, Eq. 6: M^T dY with dense X), and
// U^T Y of the closed form W* = V S^+ U^T Y (Thm. 1).
//
// A is n x p (p <= 128) and B is n x q (q <= 160), both FP32 row-major.  Each
// CTA reduces a contiguous range of rows, 32 rows (one 128-byte K step of
// FP32) at a time: the rows of A and of B are copied raw into a ring of
// shared-memory stages (one bulk copy per operand when its rows are
// contiguous, else 16-byte cp.async pieces), then producer warps write each
// chunk transposed as two K-major operand tiles (128-byte swizzle), split
// into TF32 hi and lo parts: row m of tile A is column m of A over the
// chunk's rows, row c of tile B is column c of B.  One MMA shape covers the
// product: M = 128 (columns of A), N = round16(q) (columns of B), 3xTF32
// (hi*hi + hi*lo + lo*hi).  As in the Gram kernel of CholeskyQR, each
// 384-row segment is accumulated in tensor memory (two buffers, alternating)
// and eight epilogue warps add it with round-to-nearest FP32 additions into
// the CTA's partial held in registers (thread = one row of C, half of its
// columns); the CTA's partial is written once, in FP64, and the caller adds
// the partials in a fixed order (deterministic).
#include <mutex>

#include "internal.h"
#include "tc_common.cuh"

namespace isvd {
namespace {

using namespace tc;

constexpr int kProdWarps = 7;
constexpr int kProd = kProdWarps * 32;
constexpr int kMmaWarp = kProdWarps;
constexpr int kEpiWarp0 = kProdWarps + 1;
constexpr int kEpiThreads = 256;
constexpr int kThreads = kProd + 32 + kEpiThreads;
constexpr int kHalfBlocks = 5;     // 16-column blocks per epilogue half (q <= 160)
constexpr int kBK = 32;            // rows per chunk (128 bytes of FP32 K per tile row)
constexpr int kTileStages = 2;
constexpr int kRawStages = 2;
constexpr int kMaxP = 128, kMaxQ = 160;
constexpr int kTileA = 128 * 128;  // bytes of one A tile (128 rows of 128 bytes)
constexpr int kTmemCols = 512;
constexpr int kAccCols = 256;
constexpr int kSegRows = 384;
constexpr int kF = kSegRows / kBK;  // chunks per segment
constexpr int kMaxTasks = ((kMaxP + kMaxQ) * 8 + kProd - 1) / kProd;

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void producer_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kProd) : "memory"); }

struct AbShape {
  int pa, pb;      // raw row pitches in elements (round8 of p and q)
  int n1;          // MMA N = round16(q)
  int tile_b;      // bytes of one B tile (n1 rows of 128 bytes)
  int stage;       // bytes of one tile stage (A hi, A lo, B hi, B lo)
  int raw;         // bytes of one raw stage (kBK rows of A, then kBK rows of B)
};

__host__ __device__ inline AbShape ab_shape(int p, int q) {
  AbShape s;
  s.pa = (p + 7) & ~7;
  s.pb = (q + 7) & ~7;
  s.n1 = (q + 15) & ~15;
  s.tile_b = s.n1 * 128;
  s.stage = 2 * kTileA + 2 * s.tile_b;
  s.raw = kBK * (s.pa + s.pb) * 4;
  return s;
}

size_t gram_ab_smem(int p, int q) {
  const AbShape s = ab_shape(p, q);
  return (size_t)kTileStages * s.stage + (size_t)kRawStages * s.raw + 1024;
}

__global__ void __launch_bounds__(kThreads, 1)
    gram_ab_tc_kernel(const float *__restrict__ A, int64_t lda, int32_t p, const float *__restrict__ B, int64_t ldb,
                      int32_t q, int64_t rows, int64_t rows_per_cta, int32_t bulk_a, int32_t bulk_b,
                      double *__restrict__ partial, int32_t *err) {
  const AbShape sh = ab_shape(p, q);
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t full[kTileStages], empty[kTileStages], seg_full[2], seg_free[2], raw_full[kRawStages];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  unsigned char *sm = smraw + ((1024u - (smem_u32(smraw) & 1023u)) & 1023u);
  unsigned char *tiles = sm;                                  // [kTileStages][A hi, A lo, B hi, B lo]
  unsigned char *raw = sm + (size_t)kTileStages * sh.stage;   // [kRawStages][A rows | B rows]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
  const int64_t r1 = min(rows, r0 + rows_per_cta);
  const int nchunks = r1 > r0 ? (int)((r1 - r0 + kBK - 1) / kBK) : 0;
  const int nseg = (nchunks + kF - 1) / kF;

  for (int i = tid; i < kTileStages * sh.stage / 16; i += blockDim.x)
    reinterpret_cast<uint4 *>(tiles)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    for (int s = 0; s < kTileStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&seg_full[b], 1);
      mbar_init(&seg_free[b], kEpiThreads);
    }
    // a raw stage completes on the bulk copies' bytes (one arrival by thread 0)
    // plus, for an operand copied in pieces, every producer's cp.async arrival
    const int arrivals = ((bulk_a || bulk_b) ? 1 : 0) + ((bulk_a && bulk_b) ? 0 : kProd);
    for (int s = 0; s < kRawStages; ++s) mbar_init(&raw_full[s], arrivals);
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
    int issued = 0;
    auto issue = [&](int c) {
      if (c >= nchunks) return;
      unsigned char *rb = raw + (size_t)(c % kRawStages) * sh.raw;
      unsigned char *rbb = rb + (size_t)kBK * sh.pa * 4;
      const int64_t row0 = r0 + (int64_t)c * kBK;
      const int valid = (int)((r1 - row0) < kBK ? (r1 - row0) : kBK);
      uint64_t *bar = &raw_full[c % kRawStages];
      if ((bulk_a || bulk_b) && tid == 0) {
        const uint32_t ba = bulk_a ? (uint32_t)valid * sh.pa * 4 : 0u;
        const uint32_t bb = bulk_b ? (uint32_t)valid * sh.pb * 4 : 0u;
        mbar_expect_tx(bar, ba + bb);
        if (bulk_a) bulk_g2s(smem_u32(rb), A + (size_t)row0 * lda, ba, bar);
        if (bulk_b) bulk_g2s(smem_u32(rbb), B + (size_t)row0 * ldb, bb, bar);
      }
      if (!(bulk_a && bulk_b)) {
        // the operands without contiguous rows, in 16-byte pieces
        for (int op = 0; op < 2; ++op) {
          if (op == 0 ? bulk_a : bulk_b) continue;
          const float *src = op == 0 ? A : B;
          const int64_t ld = op == 0 ? lda : ldb;
          const int pitch = op == 0 ? sh.pa : sh.pb;
          const int width = op == 0 ? p : q;
          unsigned char *dst = op == 0 ? rb : rbb;
          const int pieces = (width * 4 + 15) / 16;
          for (int t = tid; t < valid * pieces; t += kProd) {
            const int rr = t / pieces, pc = t - rr * pieces;
            cp_async16(smem_u32(dst + (size_t)rr * pitch * 4 + pc * 16), src + (size_t)(row0 + rr) * ld + pc * 4);
          }
        }
        cp_async_arrive_noinc(bar);
      }
      issued = c + 1;
    };
    // task (column m of A or c of B, kq): 4 rows (16 bytes of K) of the column,
    // the same for every chunk: offsets computed once
    uint32_t src_off[kMaxTasks], dst_off[kMaxTasks];
    int row_of[kMaxTasks];
    int ntask = 0;
    const int ncol = p + q;
#pragma unroll
    for (int i = 0; i < kMaxTasks; ++i) {
      const int t = tid + i * kProd;
      const int m = t % ncol, kq = t / ncol;
      row_of[i] = 4 * kq;
      if (m < p) {  // A column m -> tile A row m
        src_off[i] = (uint32_t)(row_of[i] * sh.pa * 4 + m * 4);
        dst_off[i] = sw128(m, 16 * kq);
      } else {  // B column c -> tile B row c
        const int cc = m - p;
        src_off[i] = (uint32_t)(kBK * sh.pa * 4 + row_of[i] * sh.pb * 4 + cc * 4);
        dst_off[i] = (uint32_t)(2 * kTileA) + sw128(cc, 16 * kq);
      }
      if (t < ncol * 8) ntask = i + 1;
    }
    int c = 0;
    for (int j = 0; j < kRawStages - 1; ++j) issue(j);
    for (; c < nchunks; ++c) {
      issue(c + kRawStages - 1);
      const int s = c % kTileStages;
      bool ok = mbar_wait(&raw_full[c % kRawStages], (uint32_t)((c / kRawStages) & 1));
      if (tid == 0 && c >= kTileStages && !mbar_wait(&empty[s], ((c / kTileStages) & 1) ^ 1)) ok = false;
      if (!ok) {
        abort_flag = 1;
        if (err) atomicExch(err, 1);
      }
      producer_bar();  // chunk c is in shared memory; tile stage s is free
      if (abort_flag) break;
      const unsigned char *rb = raw + (size_t)(c % kRawStages) * sh.raw;
      const int64_t row0 = r0 + (int64_t)c * kBK;
      const int valid = (int)((r1 - row0) < kBK ? (r1 - row0) : kBK);
      unsigned char *st = tiles + (size_t)s * sh.stage;
#pragma unroll
      for (int i = 0; i < kMaxTasks; ++i) {
        if (i >= ntask) break;
        const unsigned char *src = rb + src_off[i];
        const int t = tid + i * kProd;
        const int rs = (t % ncol) < p ? sh.pa * 4 : sh.pb * 4;  // raw row pitch of the task's operand
        const int rr0 = row_of[i];
        float hi[4], lo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float x = (valid == kBK || rr0 + j < valid) ? *reinterpret_cast<const float *>(src + j * rs) : 0.f;
          split_tf32(x, hi[j], lo[j]);
        }
        // hi parts at dst_off, lo parts one tile further (A lo after A hi, B lo after B hi)
        const uint32_t lo_off = dst_off[i] < (uint32_t)(2 * kTileA) ? (uint32_t)kTileA : (uint32_t)sh.tile_b;
        *reinterpret_cast<float4 *>(st + dst_off[i]) = make_float4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<float4 *>(st + dst_off[i] + lo_off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
      }
      fence_async_shared();
      producer_bar();
      if (tid == 0) mbar_arrive(&full[s]);
    }
    for (int j = c; j < issued; ++j) mbar_wait(&raw_full[j % kRawStages], (uint32_t)((j / kRawStages) & 1));
    cp_async_wait<0>();
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t id = idesc(2u, 128, sh.n1);
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % kTileStages;
        const int seg = c / kF, b = seg & 1, cs = c - seg * kF;
        if (cs == 0 && seg >= 2 && !mbar_wait(&seg_free[b], (uint32_t)(((seg >> 1) - 1) & 1))) {
          if (err) atomicExch(err, 1);
          abort_flag = 1;
          break;
        }
        if (abort_flag || !mbar_wait(&full[s], (c / kTileStages) & 1)) {
          if (err) atomicExch(err, 1);
          abort_flag = 1;
          break;
        }
        fence_after();
        const uint32_t d = tmem + (uint32_t)(b * kAccCols);
        const uint32_t ahi = smem_u32(tiles + (size_t)s * sh.stage);
        const uint32_t alo = ahi + kTileA;
        const uint32_t bhi = ahi + 2 * kTileA;
        const uint32_t blo = bhi + sh.tile_b;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t acc = (cs > 0 || kk > 0) ? 1u : 0u;
          const uint64_t ah = desc_sw128(ahi + kk * 32, 1024), al = desc_sw128(alo + kk * 32, 1024);
          const uint64_t bh = desc_sw128(bhi + kk * 32, 1024), bl = desc_sw128(blo + kk * 32, 1024);
          mma_tf32(d, ah, bh, id, acc);
          mma_tf32(d, ah, bl, id, 1u);
          mma_tf32(d, al, bh, id, 1u);
        }
        commit(&empty[s]);
        if (cs == kF - 1 || c == nchunks - 1) commit(&seg_full[b]);
      }
    }
  } else {
    // ---------------- epilogue: segment sums -> register partial ----------------
    // thread (quarter qq, half h, lane) owns row i = 32 qq + lane of C and
    // columns [80 h, 80 h + 80)
    const int qq = warp & 3;
    const int h = (warp - kEpiWarp0) >> 2;
    const int i = qq * 32 + lane;
    const int nblk = sh.n1 / 16;
    float part[kHalfBlocks][16];
#pragma unroll
    for (int k = 0; k < kHalfBlocks; ++k)
#pragma unroll
      for (int j = 0; j < 16; ++j) part[k][j] = 0.f;
    uint32_t v[16];
    for (int seg = 0; seg < nseg; ++seg) {
      const int b = seg & 1;
      if (!mbar_wait(&seg_full[b], (uint32_t)((seg >> 1) & 1))) {
        if (err && lane == 0) atomicExch(err, 1);
        break;
      }
      fence_after();
      const uint32_t d = tmem + (uint32_t)(b * kAccCols) + ((uint32_t)(qq * 32) << 16);
#pragma unroll
      for (int k = 0; k < kHalfBlocks; ++k) {
        const int blk = h * kHalfBlocks + k;
        if (blk < nblk) {
          tmem_ld16(d + (uint32_t)(blk * 16), v);
#pragma unroll
          for (int j = 0; j < 16; ++j) part[k][j] = __fadd_rn(part[k][j], __uint_as_float(v[j]));
        }
      }
      fence_before();
      mbar_arrive(&seg_free[b]);
    }
    // the CTA's partial, row-major p x q in FP64 (zero when it had no rows)
    double *P = partial + (size_t)blockIdx.x * p * q;
    if (i < p) {
#pragma unroll
      for (int k = 0; k < kHalfBlocks; ++k) {
        const int c0 = (h * kHalfBlocks + k) * 16;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < q) P[(size_t)i * q + c0 + j] = (double)part[k][j];
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

std::once_flag g_once;
cudaError_t g_err = cudaSuccess;

}  // namespace

int32_t gram_ab_parts(int64_t rows) {
  int64_t parts = ceil_div(rows, 2 * kSegRows);
  if (parts > kNumSMs) parts = kNumSMs;
  if (parts < 1) parts = 1;
  return (int32_t)parts;
}

cudaError_t gram_ab_launch(const float *A, int64_t lda, int32_t p, const float *B, int64_t ldb, int32_t q,
                           int64_t rows, double *partial, int32_t parts, int32_t *err, bool *launched,
                           cudaStream_t s) {
  *launched = false;
  if (p < 1 || p > kMaxP || q < 1 || q > kMaxQ || rows < 1 || parts < 1 || (lda & 3) || (ldb & 3) ||
      ((uintptr_t)A & 15) || ((uintptr_t)B & 15) || lda < p || ldb < q)
    return cudaSuccess;
  std::call_once(g_once, [] {
    g_err = cudaFuncSetAttribute(gram_ab_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gram_ab_smem(kMaxP, kMaxQ));
  });
  if (g_err != cudaSuccess) return g_err;
  const AbShape sh = ab_shape(p, q);
  const int64_t rpc = round_up(ceil_div(rows, parts), kBK);
  const int32_t used = (int32_t)ceil_div(rows, rpc);
  // one bulk copy per chunk and operand when the operand's rows are contiguous
  const int32_t bulk_a = lda == sh.pa ? 1 : 0;
  const int32_t bulk_b = ldb == sh.pb ? 1 : 0;
  gram_ab_tc_kernel<<<used, kThreads, gram_ab_smem(p, q), s>>>(A, lda, p, B, ldb, q, rows, rpc, bulk_a, bulk_b,
                                                               partial, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the partials of the CTAs past the last row range are zero
  if (used < parts) {
    e = cudaMemsetAsync(partial + (size_t)used * p * q, 0, sizeof(double) * (size_t)(parts - used) * p * q, s);
    if (e != cudaSuccess) return e;
  }
  *launched = true;
  return cudaSuccess;
}

}  // namespace isvd
