// Q <- Q B on tcgen05 with B upper triangular (B = R^-1 of CholeskyQR,
// Alg. 2: Q_hat = Q (L^-1)^T, L^T = R), in place, Q n x l row-major, l <= 160;
// and the general product Out[:, n0:n0+w] = Q B[:, n0:n0+w] into another
// block (the U = Q Vo and V = Qt Uo products that close Alg. 1), in column
// slices whose B panels fit in shared memory.
//
// B stays in shared memory for the whole kernel as K-major panels (128-byte
// swizzle) of 32 (FP32) or 64 (BF16) rows of K; because B is upper
// triangular, panel p only multiplies output columns n >= first k of the
// panel, so it is stored and multiplied for those columns only (MMA N shrinks
// panel by panel, and its accumulator starts at that column).  Q is streamed in
// 128-row tiles, panel by panel, straight into the swizzled layout (row r of
// the tile = 128 bytes of row r of Q): one TMA box load per panel (the tensor
// map zero-fills columns >= l and rows past the end), or 16-byte cp.async
// pieces where the block's base or pitch rules TMA out; three panels ahead of
// the two operand stages the MMA reads.  FP32 blocks use
// 3xTF32 (A and B split into TF32 hi + lo); BF16 blocks one BF16 MMA.  The
// FP32 accumulator (128 x round16(l)) is double-buffered in tensor memory so
// the epilogue warps write tile t while tile t+1 is multiplied.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "internal.h"
#include "tc_common.cuh"

namespace isvd {
namespace {

using namespace tc;

constexpr int kProdWarps = 8;
constexpr int kProd = kProdWarps * 32;
constexpr int kMmaWarp = kProdWarps;       // warp 8
constexpr int kThreads = (kProdWarps + 1 + 4) * 32;
constexpr int kStages = 2;  // operand stages shared with the MMA warp
constexpr int kMaxSmem = 225 * 1024;  // dynamic; the static barriers take the rest of the 227 KB
constexpr int kTmemCols = 512;
constexpr int kDBufCol = 256;  // column offset of accumulator buffer 1

__device__ __forceinline__ void cp_async16_zfill(uint32_t saddr, const void *g, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(g), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void producer_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kProd) : "memory"); }

// 8 words to global memory: one 32-byte store when `aligned32` (the address
// is then a multiple of 32), else two 16-byte stores (16-byte aligned address)
__device__ __forceinline__ void st_32(void *p, bool aligned32, uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                                      uint32_t e, uint32_t f, uint32_t g, uint32_t h) {
  if (aligned32) {
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(a), "r"(b), "r"(c), "r"(d),
                 "r"(e), "r"(f), "r"(g), "r"(h)
                 : "memory");
  } else {
    reinterpret_cast<uint4 *>(p)[0] = make_uint4(a, b, c, d);
    reinterpret_cast<uint4 *>(p)[1] = make_uint4(e, f, g, h);
  }
}

template <int DT>
struct GemmCfg {
  static constexpr bool F32 = DT == DT_F32;
  static constexpr int ES = F32 ? 4 : 2;
  static constexpr int KE = F32 ? 32 : 64;  // K elements per panel (128 bytes)
  static constexpr int NT = F32 ? 2 : 1;
  static constexpr int STAGE = NT * 128 * 128;  // bytes per A stage
};

// Panel p of B holds K rows [p*KE, p*KE + KE).  Triangular B: output columns
// n in [p*KE, N1), np(p) = N1 - p*KE rows of 128 bytes at byte offset
// bo(p) = 128 * sum_{q<p} np(q); general B: all N1 columns in every panel.
struct Layout {
  int KE, KP, N1, tri, bbytes;
  __host__ __device__ int n_first(int p) const { return tri ? p * KE : 0; }
  __host__ __device__ int np(int p) const { return N1 - n_first(p); }
  __host__ __device__ int bo(int p) const { return tri ? 128 * (p * N1 - KE * p * (p - 1) / 2) : 128 * p * N1; }
};

// K = l; w output columns (w = l for the triangular in-place product)
template <int DT>
__host__ __device__ Layout make_layout(int l, int w, int tri) {
  using C = GemmCfg<DT>;
  Layout L{};
  L.KE = C::KE;
  L.KP = (l + C::KE - 1) / C::KE;
  L.N1 = (w + 15) & ~15;
  L.tri = tri;
  L.bbytes = L.bo(L.KP);
  return L;
}

// The output block: Out[row][c] for c < w, from B's columns n0 + c.
struct GemmOut {
  void *out;
  int64_t ldo;
  int32_t n0, w, tri;
  int32_t sub;  // FP32 only: out <- out - Q B (the output block read back in the epilogue)
  // nullable: column sums of the stored output (the all-ones projection 1^T Q
  // of the next product), FP64 partials [gridDim.x * 4][cs_ld], one per CTA
  // and TMEM lane quarter
  double *colsum;
  int32_t cs_ld;
};

// Sum over the 32 lanes of each of x[0..31], lane c receiving column c's
// sum: five halving exchanges (16 + 8 + 4 + 2 + 1 shuffles).
__device__ __forceinline__ float lane_column_sum(float x[32], int lane) {
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool upper = (lane & h) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float keep = upper ? x[h + i] : x[i];
      const float give = upper ? x[i] : x[h + i];
      x[i] = keep + __shfl_xor_sync(0xffffffffu, give, h);
    }
  }
  return x[0];
}

// kRaw: raw panels in flight (refilled by the producers alone); 3 where the
// shared memory allows, else 2.
template <int DT, int kRaw>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_tc_kernel(const void *__restrict__ Qv, int64_t ldq, int64_t rows, int32_t l, const float *__restrict__ B,
                   int64_t ldb, const GemmOut o, const __grid_constant__ CUtensorMap tmap, int32_t use_tma,
                   const int32_t *gate_state, int32_t gate_pass, int32_t *err_state) {
  using C = GemmCfg<DT>;
  if (gate_state && gate_pass > 2 && gate_state[0] + 2 < gate_pass) return;
  const Layout L = make_layout<DT>(l, o.w, o.tri);
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], dfull[2], dfree[2], raw_full[kRaw], raw_empty[kRaw];
  // BF16 panels need no transform: with TMA (zero-filled padding) the MMA reads
  // them straight from the raw stage, which it releases itself
  const bool direct = !C::F32 && use_tma;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  unsigned char *sm = smraw + ((1024u - (tc::smem_u32(smraw) & 1023u)) & 1023u);
  unsigned char *bhi = sm;
  unsigned char *blo = sm + L.bbytes;                         // F32 only
  unsigned char *astage = sm + C::NT * L.bbytes;              // [kStages][NT][16 KB]
  unsigned char *rawring = astage + (size_t)kStages * C::STAGE;  // [kRaw][16 KB]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntiles = (rows + 127) / 128;
  const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t G = my_tiles * L.KP;

  // B panels: element (k, n0 + n) of B, k in panel p, n from n_first(p), stored K-major
  for (int p = 0; p < L.KP; ++p) {
    const int k0 = p * C::KE;
    for (int idx = tid; idx < L.np(p) * C::KE; idx += blockDim.x) {
      const int nn = idx / C::KE, kk = idx - nn * C::KE;
      const int n = L.n_first(p) + nn, k = k0 + kk;
      const float x = (k < l && n < o.w && (!o.tri || k <= n)) ? B[(size_t)k * ldb + o.n0 + n] : 0.f;
      const uint32_t off = L.bo(p) + sw128(nn, kk * C::ES);
      if (C::F32) {
        float hi, lo;
        split_tf32(x, hi, lo);
        *reinterpret_cast<float *>(bhi + off) = hi;
        *reinterpret_cast<float *>(blo + off) = lo;
      } else {
        *reinterpret_cast<__nv_bfloat16 *>(bhi + off) = __float2bfloat16_rn(x);
      }
    }
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);  // one arrive after the producers' barrier
      mbar_init(&empty[s], 1);
    }
    for (int d = 0; d < 2; ++d) {
      mbar_init(&dfull[d], 1);
      mbar_init(&dfree[d], 128);
    }
    for (int r = 0; r < kRaw; ++r) {
      mbar_init(&raw_full[r], 1);  // TMA: one expect_tx arrive + the box bytes
      mbar_init(&raw_empty[r], 1);  // direct form: the MMA's commit
    }
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
  const char *Q = reinterpret_cast<const char *>(Qv);

  if (warp < kProdWarps) {
    // ---------------- producers: stream A panels ----------------
    // Raw panels land in a ring of kRaw stages (cp.async, swizzled layout) that
    // the producers refill as soon as they have transformed a panel, so loads
    // run ahead of the MMA; the transform writes the operand stage (TF32 hi / lo
    // or BF16 with padding columns zeroed) once the MMA has released it.
    auto tile_row0 = [&](int64_t lt) { return ((int64_t)blockIdx.x + lt * gridDim.x) * 128; };
    auto issue = [&](int64_t g) {
      if (g < G && use_tma) {
        if (tid == 0) {
          const int64_t lt = g / L.KP;
          const int p = (int)(g - lt * L.KP);
          unsigned char *rb = rawring + (size_t)(g % kRaw) * (128 * 128);
          mbar_expect_tx(&raw_full[g % kRaw], 128 * 128);
          tma_load_2d(smem_u32(rb), &tmap, p * C::KE, (int32_t)tile_row0(lt), &raw_full[g % kRaw]);
        }
      } else if (g < G) {
        const int64_t lt = g / L.KP;
        const int p = (int)(g - lt * L.KP);
        unsigned char *rb = rawring + (size_t)(g % kRaw) * (128 * 128);
        const int64_t r0 = tile_row0(lt);
        for (int t = tid; t < 128 * 8; t += kProd) {  // 128 rows x 8 pieces of 16 bytes
          const int r = t >> 3, q = t & 7;
          const int64_t row = r0 + r;
          const int64_t colb = (int64_t)p * 128 + q * 16;   // byte offset in the row
          const bool ok = row < rows && colb < ldq * C::ES;
          const char *src = ok ? Q + ((size_t)row * ldq) * C::ES + colb : Q;
          cp_async16_zfill(smem_u32(rb + sw128(r, q * 16)), src, ok ? 16u : 0u);
        }
      }
      cp_async_commit();  // one group per panel (empty past the end) keeps the wait count fixed
    };
    // this thread's four 16-byte pieces of a panel: (row t / 8, chunk t % 8)
    // for t = tid + i kProd; the same swizzled offsets in every panel
    static_assert(128 * 8 == 4 * kProd, "four 16-byte pieces of a panel per producer thread");
    uint32_t poff[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int t = tid + i * kProd;
      poff[i] = sw128(t >> 3, (t & 7) * 16);
    }
    auto transform = [&](int64_t g) {
      const int s = (int)(g % kStages);
      const int p = (int)(g % L.KP);
      const unsigned char *rb = rawring + (size_t)(g % kRaw) * (128 * 128);
      unsigned char *ahi = astage + (size_t)s * C::STAGE;
      unsigned char *alo = ahi + 128 * 128;
      // padding columns (>= l) never enter the product: TMA fills them with
      // zeros, the cp.async pieces are cleared here
      const bool clear = !use_tma && (p + 1) * C::KE > l;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint32_t off = poff[i];
        const int k0 = p * C::KE + (((tid + i * kProd) & 7) * (16 / C::ES));  // first column of this piece
        if (C::F32) {
          const float4 v = *reinterpret_cast<const float4 *>(rb + off);
          float x[4] = {v.x, v.y, v.z, v.w}, hi[4], lo[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (clear && k0 + j >= l) x[j] = 0.f;
            split_tf32(x[j], hi[j], lo[j]);
          }
          *reinterpret_cast<float4 *>(ahi + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<float4 *>(alo + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        } else {
          uint4 v = *reinterpret_cast<const uint4 *>(rb + off);
          if (clear && k0 + 8 > l) {
            unsigned short *h = reinterpret_cast<unsigned short *>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j)
              if (k0 + j >= l) h[j] = 0;
          }
          *reinterpret_cast<uint4 *>(ahi + off) = v;
        }
      }
    };
    if (direct) {
      // one thread streams the panels into the raw ring as the MMA frees it
      if (tid == 0) {
        int64_t g = 0;
        for (; g < G; ++g) {
          if (g >= kRaw && !mbar_wait(&raw_empty[g % kRaw], (uint32_t)(((g / kRaw) - 1) & 1))) {
            abort_flag = 1;
            if (err_state) atomicExch(&err_state[2], 1);
            break;
          }
          issue(g);
        }
        // after an abort, let the boxes already requested land before the CTA exits
        for (int64_t j = std::max<int64_t>(0, g - kRaw); j < g; ++j)
          mbar_wait(&raw_full[j % kRaw], (uint32_t)((j / kRaw) & 1));
      }
    } else {
    for (int64_t g = 0; g < kRaw - 1; ++g) issue(g);
    int64_t g = 0;
    for (; g < G; ++g) {
      issue(g + kRaw - 1);           // into the raw stage transformed in the previous iteration
      bool ok = true;
      if (use_tma) ok = mbar_wait(&raw_full[g % kRaw], (uint32_t)((g / kRaw) & 1));  // the box landed
      else cp_async_wait<kRaw - 1>();  // this thread's copies of panel g have landed
      const int s = (int)(g % kStages);
      if (tid == 0 && g >= kStages && !mbar_wait(&empty[s], (uint32_t)(((g / kStages) & 1) ^ 1))) ok = false;
      if (!ok) {
        abort_flag = 1;
        if (err_state) atomicExch(&err_state[2], 1);
      }
      producer_bar();  // panel g is in shared memory; operand stage s is free
      if (abort_flag) break;
      transform(g);
      fence_async_shared();
      producer_bar();  // the operand stage is written (and the raw stage of panel g may be refilled)
      if (tid == 0) mbar_arrive(&full[s]);
    }
    // after an abort, let the boxes already requested land before the CTA exits
    if (use_tma)
      for (int64_t j = g; j < std::min<int64_t>(G, g + kRaw); ++j)
        mbar_wait(&raw_full[j % kRaw], (uint32_t)((j / kRaw) & 1));
    cp_async_wait<0>();
    }
  } else if (warp == kMmaWarp) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      const uint32_t fmt = C::F32 ? 2u : 1u;
      for (int64_t lt = 0; lt < my_tiles && !abort_flag; ++lt) {
        const int d = (int)(lt & 1);
        if (lt >= 2 && !mbar_wait(&dfree[d], (uint32_t)(((lt >> 1) & 1) ^ 1))) {
          if (err_state) atomicExch(&err_state[2], 1);
          abort_flag = 1;
          break;
        }
        fence_after();
        const uint32_t dcol = tmem + (d ? kDBufCol : 0);
        for (int p = 0; p < L.KP; ++p) {
          const int64_t g = lt * L.KP + p;
          const int s = (int)(g % kStages);
          const bool ok = direct ? mbar_wait(&raw_full[g % kRaw], (uint32_t)((g / kRaw) & 1))
                                 : mbar_wait(&full[s], (uint32_t)((g / kStages) & 1));
          if (!ok) {
            if (err_state) atomicExch(&err_state[2], 1);
            abort_flag = 1;
            break;
          }
          fence_after();
          const uint32_t id = idesc(fmt, 128, L.np(p));
          const uint32_t ahi = direct ? smem_u32(rawring + (size_t)(g % kRaw) * (128 * 128))
                                      : smem_u32(astage + (size_t)s * C::STAGE);
          const uint32_t alo = ahi + 128 * 128;
          const uint32_t b_hi = smem_u32(bhi + L.bo(p)), b_lo = smem_u32(blo + L.bo(p));
          const uint32_t dp = dcol + L.n_first(p);  // accumulator columns from n_first(p)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint32_t acc = (p > 0 || kk > 0) ? 1u : 0u;
            const uint64_t da = desc_sw128(ahi + kk * 32, 1024), db = desc_sw128(b_hi + kk * 32, 1024);
            if (C::F32) {
              mma_tf32(dp, da, db, id, acc);
              mma_tf32(dp, da, desc_sw128(b_lo + kk * 32, 1024), id, 1u);
              mma_tf32(dp, desc_sw128(alo + kk * 32, 1024), db, id, 1u);
            } else {
              mma_bf16(dp, da, db, id, acc);
            }
          }
          commit(direct ? &raw_empty[g % kRaw] : &empty[s]);
        }
        commit(&dfull[d]);
      }
    }
  } else {
    // ---------------- epilogue: TMEM -> output rows ----------------
    const int sub = warp & 3;  // TMEM lane quarter of this warp
    const int r = sub * 32 + lane;
    char *Out = reinterpret_cast<char *>(o.out);
    // every row start is 32-byte aligned (the column offsets below are multiples of 32 bytes)
    const bool v32 = ((uintptr_t)Out & 31) == 0 && ((o.ldo * C::ES) & 31) == 0;
    double cacc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // column sums (chunk cb / 32, column cb + lane)
    for (int64_t lt = 0; lt < my_tiles; ++lt) {
      const int d = (int)(lt & 1);
      if (!mbar_wait_sleep(&dfull[d], (uint32_t)((lt >> 1) & 1), 256)) {
        if (err_state && lane == 0) atomicExch(&err_state[2], 1);
        break;
      }
      fence_after();
      const int64_t row = ((int64_t)blockIdx.x + lt * gridDim.x) * 128 + r;
      uint32_t v[32];
      for (int cb = 0; cb < L.N1; cb += 32) {
        tmem_ld32(tmem + ((uint32_t)(sub * 32) << 16) + (d ? kDBufCol : 0) + cb, v);
        if (row < rows) {
          char *dst = Out + ((size_t)row * o.ldo + cb) * C::ES;
          // 32-byte stores (a whole L2 sector each) where every row starts
          // on a 32-byte boundary, else 16-byte pairs (the row pitch is a
          // multiple of 8 elements); element stores for a ragged tail
          const int n = min(32, o.w - cb);
          if (C::F32) {
            if (o.sub) {
#pragma unroll
              for (int j = 0; j < 32; j += 4) {
                if (j + 4 <= n) {
                  const float4 old = *reinterpret_cast<const float4 *>(dst + j * 4);
                  v[j] = __float_as_uint(old.x - __uint_as_float(v[j]));
                  v[j + 1] = __float_as_uint(old.y - __uint_as_float(v[j + 1]));
                  v[j + 2] = __float_as_uint(old.z - __uint_as_float(v[j + 2]));
                  v[j + 3] = __float_as_uint(old.w - __uint_as_float(v[j + 3]));
                } else {
#pragma unroll
                  for (int t = 0; t < 4; ++t)
                    if (j + t < n)
                      v[j + t] = __float_as_uint(reinterpret_cast<const float *>(dst)[j + t] - __uint_as_float(v[j + t]));
                }
              }
            }
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
              if (j + 8 <= n) {
                st_32(dst + j * 4, v32, v[j], v[j + 1], v[j + 2], v[j + 3], v[j + 4], v[j + 5], v[j + 6], v[j + 7]);
              } else {
#pragma unroll
                for (int t = 0; t < 8; ++t)
                  if (j + t < n) reinterpret_cast<float *>(dst)[j + t] = __uint_as_float(v[j + t]);
              }
            }
          } else {
            uint32_t w[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) {
              const __nv_bfloat162 h = __floats2bfloat162_rn(__uint_as_float(v[2 * t]), __uint_as_float(v[2 * t + 1]));
              w[t] = *reinterpret_cast<const uint32_t *>(&h);
            }
#pragma unroll
            for (int j = 0; j < 32; j += 16) {
              const int t0 = j / 2;
              if (j + 16 <= n) {
                st_32(dst + j * 2, v32, w[t0], w[t0 + 1], w[t0 + 2], w[t0 + 3], w[t0 + 4], w[t0 + 5], w[t0 + 6],
                      w[t0 + 7]);
              } else {
#pragma unroll
                for (int t = 0; t < 16; ++t)
                  if (j + t < n)
                    reinterpret_cast<__nv_bfloat16 *>(dst)[j + t] = __float2bfloat16_rn(__uint_as_float(v[j + t]));
              }
            }
          }
        }
        if (o.colsum) {
          // the values as stored (BF16 rounded), rows past the end and
          // columns past w as zero
          const int n = min(32, o.w - cb);
          float x[32];
#pragma unroll
          for (int t = 0; t < 32; ++t) {
            float y = __uint_as_float(v[t]);
            if (!C::F32) y = __bfloat162float(__float2bfloat16_rn(y));
            x[t] = (row < rows && t < n) ? y : 0.f;
          }
          const float cs = lane_column_sum(x, lane);
#pragma unroll
          for (int k = 0; k < 5; ++k)
            if (k == cb / 32) cacc[k] += (double)cs;
        }
      }
      fence_before();
      mbar_arrive(&dfree[d]);
    }
    if (o.colsum)
      for (int cb = 0; cb < L.N1; cb += 32)
        if (cb + lane < o.w) {
          double c = 0.0;
#pragma unroll
          for (int k = 0; k < 5; ++k)
            if (k == cb / 32) c = cacc[k];
          o.colsum[((size_t)blockIdx.x * 4 + sub) * o.cs_ld + cb + lane] = c;
        }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

template <int DT>
size_t gemm_tc_smem(int32_t l, int32_t w, int32_t tri, int raw) {
  using C = GemmCfg<DT>;
  const Layout L = make_layout<DT>(l, w, tri);
  return (size_t)C::NT * L.bbytes + (size_t)kStages * C::STAGE + (size_t)raw * 128 * 128 + 1024;
}

std::once_flag g_once;
cudaError_t g_err = cudaSuccess;

}  // namespace

cudaError_t gemm_tc_init() {
  std::call_once(g_once, [] {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *fn) {
      if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
    };
    set((const void *)gemm_tc_kernel<DT_F32, 2>);
    set((const void *)gemm_tc_kernel<DT_F32, 3>);
    set((const void *)gemm_tc_kernel<DT_BF16, 2>);
    set((const void *)gemm_tc_kernel<DT_BF16, 3>);
    g_err = e;
  });
  return g_err;
}

namespace {

// cuTensorMapEncodeTiled from the driver (no link-time dependency on it)
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Tensor map of Q (rows x l, pitch ldq) with 128-byte-swizzled boxes of one
// panel (128 bytes of K) x 128 rows; false where TMA cannot be used (base not
// 16-byte aligned, pitch not a multiple of 16 bytes, no driver entry point).
template <int DT>
bool make_tmap(CUtensorMap *m, const void *Q, int64_t ldq, int64_t rows, int32_t l) {
  using C = GemmCfg<DT>;
  memset(m, 0, sizeof *m);
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn || ((uintptr_t)Q & 15) || ((ldq * C::ES) & 15) || rows < 1 || rows > (int64_t)INT32_MAX) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)l, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ldq * C::ES)};
  const cuuint32_t box[2] = {(cuuint32_t)C::KE, 128u};
  const cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = fn(m, C::F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                        const_cast<void *>(Q), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// One launch per column slice of the output; false when no slice fits.
template <int DT>
bool launch_gemm(const void *Q, int64_t ldq, int64_t rows, int32_t l, const float *B, int64_t ldb, GemmOut o,
                 PassGate g, cudaStream_t s) {
  using C = GemmCfg<DT>;
  int32_t *err = const_cast<int32_t *>(g.state);
  const int64_t ntiles = (rows + 127) / 128;
  const int grid = (int)std::min<int64_t>(ntiles, kNumSMs);
  CUtensorMap tmap;
  const int32_t tma = make_tmap<DT>(&tmap, Q, ldq, rows, l) ? 1 : 0;
  // widest slice (a multiple of 16 columns) whose B panels fit beside 2 raw stages
  int32_t wc = o.w;
  if (!o.tri)
    while (wc > 16 && gemm_tc_smem<DT>(l, wc, 0, 2) > (size_t)kMaxSmem) wc = ((wc - 1) & ~15);
  if (gemm_tc_smem<DT>(l, wc, o.tri, 2) > (size_t)kMaxSmem) return false;
  for (int32_t c0 = 0; c0 < o.w; c0 += wc) {
    GemmOut os = o;
    os.n0 = o.n0 + c0;
    os.w = std::min(wc, o.w - c0);
    os.out = reinterpret_cast<char *>(o.out) + (size_t)c0 * C::ES;
    const size_t s3 = gemm_tc_smem<DT>(l, os.w, os.tri, 3);
    if (s3 <= (size_t)kMaxSmem)
      gemm_tc_kernel<DT, 3><<<grid, kThreads, s3, s>>>(Q, ldq, rows, l, B, ldb, os, tmap, tma, g.state, g.pass, err);
    else
      gemm_tc_kernel<DT, 2><<<grid, kThreads, gemm_tc_smem<DT>(l, os.w, os.tri, 2), s>>>(
          Q, ldq, rows, l, B, ldb, os, tmap, tma, g.state, g.pass, err);
  }
  return true;
}

}  // namespace

int32_t gemm_colsum_parts(int64_t rows) {
  const int64_t ntiles = (rows + 127) / 128;
  return 4 * (int32_t)std::max<int64_t>(1, std::min<int64_t>(ntiles, kNumSMs));
}

namespace {
// out[c] = (float) sum over parts of partial[part][c], c < b; columns
// b..ldc-1 zero.  One warp per column: lane t adds parts t, t + 32, ... in
// order, then a fixed shuffle tree (deterministic).
__global__ void colsum_reduce_kernel(const double *__restrict__ partial, int32_t parts, int32_t ld, int32_t b,
                                     int32_t ldc, float *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= ldc) return;
  double s = 0.0;
  if (c < b)
    for (int p = lane; p < parts; p += 32) s += partial[(size_t)p * ld + c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[c] = (float)s;
}
}  // namespace

cudaError_t colsum_reduce_launch(const double *partial, int32_t parts, int32_t ld, int32_t b, int32_t ldc, float *out,
                                 cudaStream_t s) {
  colsum_reduce_kernel<<<(unsigned)std::max(1, (ldc + 7) / 8), 256, 0, s>>>(partial, parts, ld, b, ldc, out);
  return cudaGetLastError();
}

cudaError_t gemm_tri_inplace_launch(void *Q, int64_t ldq, int dtype, int64_t rows, int32_t l, const float *B,
                                    int64_t ldb, PassGate g, cudaStream_t s, double *colsum) {
  cudaError_t e = gemm_tc_init();
  if (e != cudaSuccess) return e;
  const GemmOut o{Q, ldq, 0, l, 1, 0, colsum, l};
  const bool ok = dtype == DT_F32 ? launch_gemm<DT_F32>(Q, ldq, rows, l, B, ldb, o, g, s)
                                  : launch_gemm<DT_BF16>(Q, ldq, rows, l, B, ldb, o, g, s);
  if (!ok) return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t gemm_tc_launch(const float *Q, int64_t ldq, int64_t rows, int32_t l, const float *B, int64_t ldb,
                           int32_t w, float *out, int64_t ldo, bool *launched, cudaStream_t s, bool subtract) {
  *launched = false;
  cudaError_t e = gemm_tc_init();
  if (e != cudaSuccess) return e;
  // 16-byte stores and TMA boxes need 16-byte rows; the caller falls back otherwise
  if (rows == 0 || w == 0 || ((uintptr_t)out & 15) || (ldo & 3) || ((uintptr_t)Q & 15) || (ldq & 3))
    return cudaSuccess;
  const GemmOut o{out, ldo, 0, w, 0, subtract ? 1 : 0, nullptr, 0};
  *launched = launch_gemm<DT_F32>(Q, ldq, rows, l, B, ldb, o, PassGate{}, s);
  return cudaGetLastError();
}

}  // namespace isvd
