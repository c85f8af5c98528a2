// Sparse x tall-skinny dense product, streamed through a shared-memory ring.
//
// Same row computation as spmm.cu (y_i = s r_i (sum_j a_ij w_j z_j + [self]
// w_i z_i) + a h_i x_i + sum_t alpha_t u_it c_t, the implicit products of
// Sec. 4 with the Horner and rank-one epilogues of Eq. 3), organised so that
// many gathers are in flight per SM without holding registers:
//   - each warp takes a fixed chunk of consecutive nonzeros (whatever the
//     rows: hub rows spread over many chunks, short rows share one);
//   - the warp walks its chunk in batches of up to 32 nonzeros (and at most
//     kRowSlots complete rows).  For batch b+1 it issues 16-byte cp.async
//     copies of every gathered row of the block (full width, one row per
//     slot) and of the axpy / self rows of the rows that end in that batch,
//     while it accumulates batch b from shared memory (double buffering);
//   - lane l owns 16-byte column chunks l and l + 32 of every row: it copies
//     exactly the bytes it later reads, so no cross-lane synchronisation is
//     needed beyond its own cp.async groups;
//   - gathers of hub columns (high degree) carry the L2 evict_last policy,
//     the rest evict_first, so that the rows most often re-read stay in L2;
//   - rows crossing a chunk boundary leave partial sums that a fix-up pass
//     adds in chunk order (deterministic); rows without nonzeros get their
//     epilogue in a separate small pass.
#include <mutex>

#include "internal.h"

namespace isvd {
namespace {

constexpr int kRowSlots = 8;               // complete rows per batch (axpy / self row slots)
constexpr int kBatch = 32;                 // nonzeros per batch
constexpr uint32_t kIdxMask = (1u << 26) - 1u;

struct RingMeta {
  float w[kBatch];
  int32_t row[kBatch];
  int32_t end[kBatch];      // row-slot index when this nonzero ends its row, else -1
  int32_t rrow[kRowSlots];  // row of each row slot
  float rs[kRowSlots];      // scalar * rowscale
  float axs[kRowSlots];     // ax_scalar * ax_rowscale
  float selfw[kRowSlots];   // weight of the self term
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp16(uint32_t dst, const void *src, uint64_t pol) {
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint64_t policy(bool keep) {
  uint64_t p;
  if (keep)
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  else
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

template <int DT>
struct RV;
template <>
struct RV<DT_F32> {
  static constexpr int VN = 4, ES = 4;
  __device__ __forceinline__ static void unpack(uint4 x, float *v) {
    v[0] = __uint_as_float(x.x);
    v[1] = __uint_as_float(x.y);
    v[2] = __uint_as_float(x.z);
    v[3] = __uint_as_float(x.w);
  }
  __device__ __forceinline__ static uint4 pack(const float *v) {
    return make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]), __float_as_uint(v[3]));
  }
  __device__ __forceinline__ static void store1(void *p, float v) { *reinterpret_cast<float *>(p) = v; }
};
template <>
struct RV<DT_BF16> {
  static constexpr int VN = 8, ES = 2;
  __device__ __forceinline__ static void unpack(uint4 x, float *v) {
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&x);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 f = __bfloat1622float2(h[k]);
      v[2 * k] = f.x;
      v[2 * k + 1] = f.y;
    }
  }
  __device__ __forceinline__ static uint4 pack(const float *v) {
    uint4 x;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&x);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
    return x;
  }
  __device__ __forceinline__ static void store1(void *p, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(p) = __float2bfloat16_rn(v);
  }
};

struct RingArgs {
  const int32_t *row_of;   // row of every nonzero
  const int32_t *tagged;   // nullable: colidx with the column's degree bucket in bits 26..30
  int32_t hot_bucket;      // gathers of columns with bucket >= hot_bucket keep L2 priority
  int64_t nnz;
  int32_t CH;
  int64_t nchunks;
  float *part;             // nchunks x 2 x pw FP32 (head / tail partial rows)
  int64_t pw;
  int32_t nch;             // 16-byte chunks per gathered row (<= 64)
  int32_t slot_bytes;      // bytes per slot (nch * 16)
  int32_t row_slots;       // kRowSlots, doubled when the self term is on
};

// Shared-memory layout of one warp: [2 buffers][kBatch + row_slots slots][slot_bytes], then [2] RingMeta.
__host__ __device__ inline size_t ring_warp_bytes(int slot_bytes, int row_slots) {
  return (size_t)2 * (kBatch + row_slots) * slot_bytes + 2 * sizeof(RingMeta);
}

// The epilogue of one complete row for the chunks this lane owns.
template <int DT>
__device__ __forceinline__ void ring_epilogue(const SpmmArgs &a, const SpmmSlab &sl, int64_t r, const float *acc,
                                              int lane, int nch, const char *axrow, const char *selfrow, float rs,
                                              float axs, float selfw, uint64_t pol_out) {
  using V = RV<DT>;
  constexpr int VN = V::VN;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int ch = lane + 32 * h;
    if (ch >= nch) break;
    const int col = ch * VN;
    if (col >= sl.width) break;
    float v[VN];
#pragma unroll
    for (int k = 0; k < VN; ++k) v[k] = acc[h * VN + k];
    if (selfrow) {
      float s[VN];
      V::unpack(*reinterpret_cast<const uint4 *>(selfrow + ch * 16), s);
#pragma unroll
      for (int k = 0; k < VN; ++k) v[k] = fmaf(selfw, s[k], v[k]);
    }
#pragma unroll
    for (int k = 0; k < VN; ++k) v[k] *= rs;
    if (axrow) {
      float x[VN];
      V::unpack(*reinterpret_cast<const uint4 *>(axrow + ch * 16), x);
#pragma unroll
      for (int k = 0; k < VN; ++k) v[k] = fmaf(axs, x[k], v[k]);
    }
    for (int t = 0; t < a.lr_rank; ++t) {
      const int tu = t - a.lr_ones_first;
      const float u = (tu < 0 || !a.lr_u) ? 1.f : __ldg(a.lr_u + (size_t)r * a.lr_ldu + tu);
      const float al = a.lr_alpha[t] * u;
      const float *c = a.lr_c + (size_t)t * a.lr_ldc + sl.col0 + col;
#pragma unroll
      for (int k = 0; k < VN; ++k)
        if (col + k < sl.width) v[k] = fmaf(al, __ldg(c + k), v[k]);
    }
    char *o = reinterpret_cast<char *>(sl.out) + ((size_t)r * sl.ldo + col) * V::ES;
    if (col + VN <= sl.width) {
      const uint4 x = V::pack(v);
      asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(o), "r"(x.x), "r"(x.y),
                   "r"(x.z), "r"(x.w), "l"(pol_out)
                   : "memory");
    } else {
      for (int k = 0; col + k < sl.width; ++k) V::store1(o + k * V::ES, v[k]);
    }
  }
}

template <int DT>
__global__ void __launch_bounds__(256) spmm_ring_kernel(const __grid_constant__ SpmmArgs a, const RingArgs g) {
  using V = RV<DT>;
  constexpr int VN = V::VN;
  extern __shared__ __align__(16) unsigned char ring_smem[];
  const SpmmSlab &sl = a.slab[0];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const size_t wbytes = ring_warp_bytes(g.slot_bytes, g.row_slots);
  unsigned char *base = ring_smem + (size_t)wi * wbytes;
  const int nslots = kBatch + g.row_slots;
  RingMeta *meta = reinterpret_cast<RingMeta *>(base + (size_t)2 * nslots * g.slot_bytes);
  auto slot = [&](int p, int q) { return base + ((size_t)p * nslots + q) * g.slot_bytes; };
  const uint64_t pol_keep = policy(true), pol_first = policy(false);
  const char *inb = reinterpret_cast<const char *>(sl.in);
  const size_t ldi_b = (size_t)sl.ldi * V::ES;
  const char *axb = reinterpret_cast<const char *>(sl.axpy);
  const size_t lda_b = (size_t)sl.lda * V::ES;
  const bool c0 = lane < g.nch, c1 = lane + 32 < g.nch;
  const int64_t nwarp = (int64_t)gridDim.x * nw;

  for (int64_t c = (int64_t)blockIdx.x * nw + wi; c < g.nchunks; c += nwarp) {
    const int64_t e0 = c * g.CH;
    const int64_t e1 = (e0 + g.CH < g.nnz) ? e0 + g.CH : g.nnz;
    const int32_t head_row = (e0 > 0 && __ldg(g.row_of + e0 - 1) == __ldg(g.row_of + e0)) ? __ldg(g.row_of + e0) : -1;

    // producer: loads the batch starting at eb into buffer p, returns its length
    auto produce = [&](int64_t eb, int p) -> int {
      RingMeta &m = meta[p];
      int nb = (int)((e1 - eb) < kBatch ? (e1 - eb) : kBatch);
      const int64_t e = eb + lane;
      const bool in = lane < nb;
      const int32_t r = in ? __ldg(g.row_of + e) : -1;
      const int32_t rn = in ? (e + 1 < g.nnz ? __ldg(g.row_of + e + 1) : -2) : -1;
      unsigned ends = __ballot_sync(0xffffffffu, in && rn != r);
      if (__popc(ends) > kRowSlots) {
        // cut the batch after its kRowSlots-th complete row
        unsigned m8 = ends;
        for (int i = 0; i < kRowSlots - 1; ++i) m8 &= m8 - 1;
        const int pos = __ffs(m8) - 1;
        nb = pos + 1;
        ends &= (pos == 31) ? 0xffffffffu : ((2u << pos) - 1u);
      }
      const bool mine = lane < nb;
      int32_t j = 0;
      bool hot = true;
      float w = 0.f;
      if (mine) {
        if (g.tagged) {
          const uint32_t t = (uint32_t)__ldg(g.tagged + e);
          j = (int32_t)(t & kIdxMask);
          hot = (int32_t)(t >> 26) >= g.hot_bucket;
        } else {
          j = __ldg(a.colidx + e);
        }
        w = a.values ? __ldg(a.values + e) : 1.f;
        if (a.colw) w *= __ldg(a.colw + j);
      }
      const bool is_end = mine && ((ends >> lane) & 1u);
      const int k = __popc(ends & ((1u << lane) - 1u));
      if (mine) {
        m.w[lane] = w;
        m.row[lane] = r;
        m.end[lane] = is_end ? k : -1;
      }
      if (is_end) {
        m.rrow[k] = r;
        m.rs[k] = a.scalar * (a.rowscale ? __ldg(a.rowscale + r) : 1.f);
        m.axs[k] = a.ax_scalar * (a.ax_rowscale ? __ldg(a.ax_rowscale + r) : 1.f);
        m.selfw[k] = a.self_term ? (a.colw ? __ldg(a.colw + r) : 1.f) : 0.f;
      }
      // gathers: every row of the batch, full width
      for (int q = 0; q < nb; ++q) {
        const int32_t jq = __shfl_sync(0xffffffffu, j, q);
        const bool hq = __shfl_sync(0xffffffffu, hot, q);
        const uint64_t pol = hq ? pol_keep : pol_first;
        const char *src = inb + (size_t)jq * ldi_b;
        const uint32_t dst = smem_addr(slot(p, q));
        if (c0) cp16(dst + lane * 16, src + lane * 16, pol);
        if (c1) cp16(dst + (lane + 32) * 16, src + (lane + 32) * 16, pol);
      }
      // axpy and self rows of the rows that end in this batch (not the head row: partial)
      const int nend = __popc(ends);
      for (int kk = 0; kk < nend; ++kk) {
        unsigned mk = ends;
        for (int i = 0; i < kk; ++i) mk &= mk - 1;
        const int src_lane = __ffs(mk) - 1;
        const int32_t rr = __shfl_sync(0xffffffffu, r, src_lane);
        if (rr == head_row) continue;
        if (axb) {
          const char *src = axb + (size_t)rr * lda_b;
          const uint32_t dst = smem_addr(slot(p, kBatch + kk));
          if (c0) cp16(dst + lane * 16, src + lane * 16, pol_first);
          if (c1) cp16(dst + (lane + 32) * 16, src + (lane + 32) * 16, pol_first);
        }
        if (a.self_term) {
          const char *src = inb + (size_t)rr * ldi_b;
          const uint32_t dst = smem_addr(slot(p, kBatch + kRowSlots + kk));
          if (c0) cp16(dst + lane * 16, src + lane * 16, pol_first);
          if (c1) cp16(dst + (lane + 32) * 16, src + (lane + 32) * 16, pol_first);
        }
      }
      cp_commit();
      return nb;
    };

    float acc[2 * VN];
#pragma unroll
    for (int k = 0; k < 2 * VN; ++k) acc[k] = 0.f;
    int32_t cur = -1;
    auto write_partial = [&](int32_t row) {
      float *pp = g.part + ((size_t)c * 2 + (row == head_row ? 0 : 1)) * g.pw + sl.col0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int ch = lane + 32 * h;
        if (ch >= g.nch) break;
#pragma unroll
        for (int k = 0; k < VN; ++k)
          if (ch * VN + k < sl.width) pp[ch * VN + k] = acc[h * VN + k];
      }
    };

    int64_t eb = e0;
    int p = 0;
    int nb = produce(eb, p);
    while (nb > 0) {
      const int64_t en = eb + nb;
      int nb_next = 0;
      if (en < e1) nb_next = produce(en, p ^ 1);
      if (nb_next > 0) cp_wait<1>();
      else cp_wait<0>();
      __syncwarp();
      const RingMeta &m = meta[p];
      for (int q = 0; q < nb; ++q) {
        const float w = m.w[q];
        if (cur < 0) cur = m.row[q];
        const unsigned char *sp = slot(p, q);
        if (c0) {
          float v[VN];
          V::unpack(*reinterpret_cast<const uint4 *>(sp + lane * 16), v);
#pragma unroll
          for (int k = 0; k < VN; ++k) acc[k] = fmaf(w, v[k], acc[k]);
        }
        if (c1) {
          float v[VN];
          V::unpack(*reinterpret_cast<const uint4 *>(sp + (lane + 32) * 16), v);
#pragma unroll
          for (int k = 0; k < VN; ++k) acc[VN + k] = fmaf(w, v[k], acc[VN + k]);
        }
        const int ek = m.end[q];
        if (ek >= 0) {
          if (cur == head_row) {
            write_partial(cur);
          } else {
            ring_epilogue<DT>(a, sl, cur, acc, lane, g.nch, axb ? (const char *)slot(p, kBatch + ek) : nullptr,
                              a.self_term ? (const char *)slot(p, kBatch + kRowSlots + ek) : nullptr, m.rs[ek],
                              m.axs[ek], m.selfw[ek], pol_first);
          }
#pragma unroll
          for (int k = 0; k < 2 * VN; ++k) acc[k] = 0.f;
          cur = -1;
        }
      }
      __syncwarp();  // buffer p is free for the batch after next
      eb = en;
      nb = nb_next;
      p ^= 1;
    }
    if (cur >= 0) write_partial(cur);  // the tail row continues in the next chunk
  }
}

// Rows split across chunks: the tail partial of their first chunk plus the head
// partials of the following chunks, in chunk order, then the epilogue.
template <int DT>
__global__ void __launch_bounds__(256) spmm_ring_fixup_kernel(const __grid_constant__ SpmmArgs a,
                                                              const int4 *__restrict__ split, int32_t nsplit,
                                                              const int32_t *__restrict__ empty, int32_t nempty,
                                                              const float *__restrict__ part, int64_t pw,
                                                              int32_t nch) {
  using V = RV<DT>;
  constexpr int VN = V::VN;
  const SpmmSlab &sl = a.slab[0];
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = (int64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t pol_first = policy(false);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < (int64_t)nsplit + nempty;
       i += nwarp) {
    const bool empty_row = i >= nsplit;
    // split rows: (row, first chunk, last chunk, 0); rows without nonzeros sum nothing
    const int4 s = empty_row ? make_int4(empty[i - nsplit], 0, -1, 0) : split[i];
    const int64_t r = s.x;
    float acc[2 * VN];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int ch = lane + 32 * h;
#pragma unroll
      for (int k = 0; k < VN; ++k) {
        const int col = ch * VN + k;
        float v = 0.f;
        if (!empty_row && ch < nch && col < sl.width) {
          v = part[((size_t)s.y * 2 + 1) * pw + sl.col0 + col];
          for (int cc = s.y + 1; cc <= s.z; ++cc) v += part[((size_t)cc * 2) * pw + sl.col0 + col];
        }
        acc[h * VN + k] = v;
      }
    }
    // axpy / self rows straight from global memory (few rows)
    const float rs = a.scalar * (a.rowscale ? __ldg(a.rowscale + r) : 1.f);
    const float axs = a.ax_scalar * (a.ax_rowscale ? __ldg(a.ax_rowscale + r) : 1.f);
    const float selfw = a.self_term ? (a.colw ? __ldg(a.colw + r) : 1.f) : 0.f;
    const char *axrow = sl.axpy ? reinterpret_cast<const char *>(sl.axpy) + (size_t)r * sl.lda * V::ES : nullptr;
    const char *selfrow = a.self_term ? reinterpret_cast<const char *>(sl.in) + (size_t)r * sl.ldi * V::ES : nullptr;
    ring_epilogue<DT>(a, sl, r, acc, lane, nch, axrow, selfrow, rs, axs, selfw, pol_first);
  }
}

template <int DT>
cudaError_t launch(const SpmmArgs &a, const ChunkPlan &cp, const RingTags &tags, float *part, int64_t pw,
                   cudaStream_t s) {
  const SpmmSlab &sl = a.slab[0];
  const int es = (int)dtype_size(DT);
  RingArgs g{};
  g.row_of = cp.row_of;
  g.nnz = cp.nnz;
  g.CH = cp.CH;
  g.nchunks = cp.nchunks;
  g.part = part;
  g.pw = pw;
  g.nch = (int32_t)ceil_div((int64_t)sl.width * es, 16);
  g.slot_bytes = g.nch * 16;
  g.row_slots = a.self_term ? 2 * kRowSlots : kRowSlots;
  g.tagged = tags.tagged;
  g.hot_bucket = 0;
  if (tags.tagged && a.cache_hints) {
    // keep the hottest columns whose rows fit the L2 budget
    double bytes = 0.0;
    int hb = 32;
    while (hb > 0 && bytes + (double)tags.hist[hb - 1] * g.slot_bytes <= (double)tags.l2_budget) {
      bytes += (double)tags.hist[hb - 1] * g.slot_bytes;
      --hb;
    }
    g.hot_bucket = hb;
  } else if (!a.cache_hints) {
    g.tagged = nullptr;
  }
  const size_t wb = ring_warp_bytes(g.slot_bytes, g.row_slots);
  int nw = (int)((size_t)kRingSmemBudget / wb);
  if (nw > 8) nw = 8;
  if (nw < 1) return cudaErrorInvalidValue;
  if (cp.nchunks > 0) {
    int64_t bx = ceil_div(cp.nchunks, nw);
    const int per_sm = (int)((size_t)kRingSmemBudget / (wb * nw));
    const int64_t cap = (int64_t)kNumSMs * (per_sm > 0 ? per_sm : 1);
    if (bx > cap) bx = cap;
    spmm_ring_kernel<DT><<<(unsigned)bx, 32 * nw, wb * nw, s>>>(a, g);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int64_t nfix = (int64_t)cp.nsplit + cp.nempty;
  if (nfix > 0) {
    int64_t bx = ceil_div(nfix, 8);
    if (bx > (int64_t)kNumSMs * 4) bx = (int64_t)kNumSMs * 4;
    spmm_ring_fixup_kernel<DT><<<(unsigned)bx, 256, 0, s>>>(a, cp.split, cp.nsplit, cp.empty, cp.nempty, part, pw,
                                                           g.nch);
  }
  return cudaGetLastError();
}

}  // namespace

int ring_max_cols(int dtype) { return dtype == DT_F32 ? 256 : 512; }

cudaError_t spmm_ring_init() {
  static cudaError_t err = cudaSuccess;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaError_t e = cudaFuncSetAttribute(spmm_ring_kernel<DT_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kRingSmemBudget);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(spmm_ring_kernel<DT_BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               kRingSmemBudget);
    err = e;
  });
  return err;
}

cudaError_t spmm_ring_launch(const SpmmArgs &a, int dtype, const ChunkPlan &cp, const RingTags &tags, float *part,
                             int64_t pw, cudaStream_t s) {
  if (a.rows == 0 || a.nslabs == 0) return cudaSuccess;
  if (a.nslabs != 1) return cudaErrorInvalidValue;
  const cudaError_t e = spmm_ring_init();
  if (e != cudaSuccess) return e;
  return dtype == DT_F32 ? launch<DT_F32>(a, cp, tags, part, pw, s) : launch<DT_BF16>(a, cp, tags, part, pw, s);
}

}  // namespace isvd
