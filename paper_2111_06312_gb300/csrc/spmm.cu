// Sparse x tall-skinny dense products with fused epilogues.
//
// Every implicit product of the paper reduces to the row computation
//     y_i = s * r_i * ( sum_{j in N(i)} a_ij w_j z_j  +  [self] w_i z_i )
//           + a * h_i * x_i  +  sum_t alpha_t u_it c_t
// (Sec. 4: only M.G and M^T.G are needed).  The Horner form of the
// polynomial sum_k c_k N^k G (Eq. 3) is a chain of such rows with the axpy
// term carrying c_k G; N = D^-1 A uses r = 1/d, N = Â uses gathered w = s
// and the self term for +I; the all-ones and low-rank corrections of Eq. 3
// are the last term, broadcast from precomputed c = V^T G (the O(n) product
// of Sec. 4's outer-product example).
//
// Layout: dense blocks are row-major.  A launch covers column slabs (grid y);
// inside a slab `group` lanes cooperate on one row, each lane owning 16 bytes
// of columns, so one gathered neighbour row is one coalesced 32..128-byte
// read.  Slabs run one after another in launch order so that the slab of
// the gathered block stays resident in L2.  A slab narrower than 32 lanes
// puts several row groups in a warp: they step through their rows together
// and take rows in degree order, so their lengths match.  Rows with more than
// `heavy_threshold` nonzeros are split into chunks whose partial sums are
// combined in chunk order (by a warp, or by a whole CTA for the largest hubs),
// so results are deterministic; the chunks run on a second stream beside the
// row kernel.
#include "internal.h"

// blocks per SM of the FP32 row kernel at high occupancy, and the nonzeros
// in flight and blocks per SM of the wide (two chunks per lane) form: build-time knobs
#ifndef ISVD_ROWS_HIGH_OCC_F32
#define ISVD_ROWS_HIGH_OCC_F32 6
#endif
#ifndef ISVD_WIDE_UNROLL
#define ISVD_WIDE_UNROLL 3
#endif
#ifndef ISVD_WIDE_MINB
#define ISVD_WIDE_MINB 4
#endif
// resident blocks per SM of the packed-slab kernel
#ifndef ISVD_SLAB_MINB_F32
#define ISVD_SLAB_MINB_F32 5
#endif
#ifndef ISVD_SLAB_MINB_BF16
#define ISVD_SLAB_MINB_BF16 5
#endif
// L2 policies of the packed-slab kernel: gathered rows of the slab
// evict_last (ISVD_SLAB_GATHER_KEEP 1) or unmarked (0); the CSR stream, the
// axpy operand and the output evict_first.  Measured on the 10^6-node
// graph at width 144: 7.94 -> 7.80 ms per FP32 apply, 5.30 -> 5.22 ms BF16
// (unmarked gathers: 7.81 and 5.36), results bit for bit the same.
#ifndef ISVD_SLAB_GATHER_KEEP
#define ISVD_SLAB_GATHER_KEEP 1
#endif

namespace isvd {
namespace {

// L2 eviction-priority policies (PTX createpolicy): gathered rows of the dense
// block are kept (evict_last); the CSR stream and the output block pass
// through (evict_first), so that the slab of the block stays in L2.
__device__ __forceinline__ uint64_t policy_keep() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_stream() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

template <bool HINT>
__device__ __forceinline__ uint4 ld16(const void *p, uint64_t pol) {
  uint4 v;
  if (HINT)
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
  else
    v = __ldg(reinterpret_cast<const uint4 *>(p));
  return v;
}

// coherent (not .nc) 16-byte load with an L2 policy: for blocks that the
// same kernel may also write (an in-place Horner accumulate)
template <bool HINT>
__device__ __forceinline__ uint4 ld16c(const void *p, uint64_t pol) {
  uint4 v;
  if (HINT)
    asm volatile("ld.global.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
  else
    v = *reinterpret_cast<const uint4 *>(p);
  return v;
}

template <bool HINT>
__device__ __forceinline__ void st16(void *p, uint4 v, uint64_t pol) {
  if (HINT)
    asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w), "l"(pol)
                 : "memory");
  else
    *reinterpret_cast<uint4 *>(p) = v;
}

template <bool HINT>
__device__ __forceinline__ int32_t ld_idx(const int32_t *p, uint64_t pol) {
  int32_t v;
  if (HINT)
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  else
    v = __ldg(p);
  return v;
}

template <int DT>
struct Vec;

template <>
struct Vec<DT_F32> {
  static constexpr int N = 4;
  static constexpr int BYTES = 4;
  __device__ __forceinline__ static void unpack(const uint4 x, float *v) {
    v[0] = __uint_as_float(x.x);
    v[1] = __uint_as_float(x.y);
    v[2] = __uint_as_float(x.z);
    v[3] = __uint_as_float(x.w);
  }
  __device__ __forceinline__ static uint4 pack(const float *v) {
    return make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]), __float_as_uint(v[3]));
  }
  __device__ __forceinline__ static void store_partial(void *p, const float *v, int valid) {
    float *q = reinterpret_cast<float *>(p);
    for (int k = 0; k < valid; ++k) q[k] = v[k];
  }
};

template <>
struct Vec<DT_BF16> {
  static constexpr int N = 8;
  static constexpr int BYTES = 2;
  __device__ __forceinline__ static void unpack(const uint4 x, float *v) {
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
  __device__ __forceinline__ static void store_partial(void *p, const float *v, int valid) {
    __nv_bfloat16 *q = reinterpret_cast<__nv_bfloat16 *>(p);
    for (int k = 0; k < valid; ++k) q[k] = __float2bfloat16_rn(v[k]);
  }
};

constexpr int kPrefetchNonzeros = 8;  // neighbour rows of the next row prefetched to L2

struct Policies {
  uint64_t keep, stream;
};

template <bool HINT>
__device__ __forceinline__ Policies make_policies() {
  Policies p{0, 0};
  if (HINT) {
    p.keep = policy_keep();
    p.stream = policy_stream();
  }
  return p;
}

struct Lane {
  int G;          // lanes per row
  int gl;         // lane within the group
  int sub;        // group index within the warp
  unsigned mask;  // lanes of this group
  int col;        // first column (within the slab) of the lane's first 16-byte chunk
  bool active;    // col < width
  int col2;       // wide slabs (two chunks per lane): first column of the second chunk
  bool active2;
};

template <int DT>
__device__ __forceinline__ Lane make_lane(const SpmmSlab &sl) {
  Lane L;
  const int lane = threadIdx.x & 31;
  L.G = sl.group;
  L.gl = lane & (L.G - 1);
  L.sub = lane / L.G;
  L.mask = (L.G == 32) ? 0xffffffffu : (((1u << L.G) - 1u) << (L.sub * L.G));
  L.col = L.gl * Vec<DT>::N;
  L.active = L.col < sl.width;
  L.col2 = (L.gl + L.G) * Vec<DT>::N;
  L.active2 = L.col2 < sl.width;
  return L;
}

// acc += sum over nonzeros e in [e0, e1) of a_e w_j in_j (slab columns of this
// lane: one 16-byte chunk, or two in wide slabs (CPL = 2), acc[c * VN + k]).
template <int DT, bool HINT, int CPL>
__device__ __forceinline__ void gather_range(const SpmmArgs &a, const SpmmSlab &sl, const Lane &L, int e0,
                                             int e1, const Policies &pol, float *acc) {
  using V = Vec<DT>;
  constexpr int VN = V::N;
  constexpr int U = CPL == 1 ? 4 : ISVD_WIDE_UNROLL;  // nonzeros per step
  const char *inb = reinterpret_cast<const char *>(sl.in) + (size_t)L.col * V::BYTES;
  const size_t off2 = (size_t)(L.col2 - L.col) * V::BYTES;
  const size_t ldb = (size_t)sl.ldi * V::BYTES;
  for (int e = e0; e < e1; e += L.G) {
    const int me = e + L.gl;
    int j = 0;
    float w = 0.f;
    if (me < e1) {
      if (HINT && a.tagged) {
        // column index in bits 0..25, degree bucket above: cold columns stream through L2
        const int32_t t = ld_idx<HINT>(a.tagged + me, pol.stream);
        j = t & ((1 << 26) - 1);
        if ((t >> 26) < sl.hot_bucket) j |= (int)0x80000000;
      } else {
        j = ld_idx<HINT>(a.colidx + me, pol.stream);
      }
      w = a.values ? __ldg(a.values + me) : 1.f;
      if (a.colw) w *= __ldg(a.colw + (j & 0x7fffffff));
    }
    const int cnt = min(L.G, e1 - e);
    int t = 0;
    for (; t + U <= cnt; t += U) {
      int jj[U];
      float ww[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        jj[u] = __shfl_sync(L.mask, j, t + u, L.G);
        ww[u] = __shfl_sync(L.mask, w, t + u, L.G);
      }
      if (L.active) {
        uint4 raw[U][CPL];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const char *src = inb + (size_t)(jj[u] & 0x7fffffff) * ldb;
          const uint64_t pl = jj[u] < 0 ? pol.stream : pol.keep;
          raw[u][0] = ld16<HINT>(src, pl);
          if (CPL == 2) raw[u][CPL - 1] = L.active2 ? ld16<HINT>(src + off2, pl) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            float v[VN];
            V::unpack(raw[u][c], v);
#pragma unroll
            for (int k = 0; k < VN; ++k) acc[c * VN + k] = fmaf(ww[u], v[k], acc[c * VN + k]);
          }
      }
    }
    for (; t < cnt; ++t) {
      const int j0 = __shfl_sync(L.mask, j, t, L.G);
      const float w0 = __shfl_sync(L.mask, w, t, L.G);
      if (L.active) {
        const char *src = inb + (size_t)(j0 & 0x7fffffff) * ldb;
        const uint64_t pl = j0 < 0 ? pol.stream : pol.keep;
        uint4 raw[CPL];
        raw[0] = ld16<HINT>(src, pl);
        if (CPL == 2) raw[CPL - 1] = L.active2 ? ld16<HINT>(src + off2, pl) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          float v[VN];
          V::unpack(raw[c], v);
#pragma unroll
          for (int k = 0; k < VN; ++k) acc[c * VN + k] = fmaf(w0, v[k], acc[c * VN + k]);
        }
      }
    }
  }
}

// The same sum for narrow slabs, whose warps hold several row groups (G < 32):
// the groups step through their rows together, to the longest row of the
// warp (maxlen, warp-uniform), so the warp issues one instruction stream
// instead of one per group; entries past a row's length (len) load nothing
// and weigh zero.  All 32 lanes must call it.
template <int DT, bool HINT, int CPL>
__device__ __forceinline__ void gather_range_grouped(const SpmmArgs &a, const SpmmSlab &sl, const Lane &L, int e0,
                                                     int len, int maxlen, const Policies &pol, float *acc) {
  using V = Vec<DT>;
  constexpr int VN = V::N;
  constexpr int U = CPL == 1 ? 4 : ISVD_WIDE_UNROLL;
  const char *inb = reinterpret_cast<const char *>(sl.in) + (size_t)L.col * V::BYTES;
  const size_t off2 = (size_t)(L.col2 - L.col) * V::BYTES;
  const size_t ldb = (size_t)sl.ldi * V::BYTES;
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
  for (int off = 0; off < maxlen; off += L.G) {
    const int me = off + L.gl;
    int j = 0;
    float w = 0.f;
    if (me < len) {
      const int e = e0 + me;
      if (HINT && a.tagged) {
        const int32_t t = ld_idx<HINT>(a.tagged + e, pol.stream);
        j = t & ((1 << 26) - 1);
        if ((t >> 26) < sl.hot_bucket) j |= (int)0x80000000;
      } else {
        j = ld_idx<HINT>(a.colidx + e, pol.stream);
      }
      w = a.values ? __ldg(a.values + e) : 1.f;
      if (a.colw) w *= __ldg(a.colw + (j & 0x7fffffff));
    }
    const int cntw = min(L.G, maxlen - off);  // warp-uniform
    for (int t = 0; t < cntw; t += U) {
      int jj[U];
      float ww[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        jj[u] = __shfl_sync(0xffffffffu, j, t + u, L.G);
        ww[u] = __shfl_sync(0xffffffffu, w, t + u, L.G);
      }
      if (L.active) {
        uint4 raw[U][CPL];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const bool ok = t + u < cntw && off + t + u < len;
          const char *src = inb + (size_t)(jj[u] & 0x7fffffff) * ldb;
          const uint64_t pl = jj[u] < 0 ? pol.stream : pol.keep;
          raw[u][0] = ok ? ld16<HINT>(src, pl) : zero;
          if (CPL == 2) raw[u][CPL - 1] = (ok && L.active2) ? ld16<HINT>(src + off2, pl) : zero;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            float v[VN];
            V::unpack(raw[u][c], v);
#pragma unroll
            for (int k = 0; k < VN; ++k) acc[c * VN + k] = fmaf(ww[u], v[k], acc[c * VN + k]);
          }
      }
    }
  }
}

template <int DT, bool HINT, int CPL>
__device__ __forceinline__ void epilogue(const SpmmArgs &a, const SpmmSlab &sl, const Lane &L, int64_t r,
                                         const Policies &pol, float *acc_all) {
  using V = Vec<DT>;
  constexpr int VN = V::N;
  const float sc = a.scalar * (a.rowscale ? __ldg(a.rowscale + r) : 1.f);
  const float as = sl.axpy ? a.ax_scalar * (a.ax_rowscale ? __ldg(a.ax_rowscale + r) : 1.f) : 0.f;
  const float ws = a.self_term ? (a.colw ? __ldg(a.colw + r) : 1.f) : 0.f;
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int col = c == 0 ? L.col : L.col2;
    if (!(c == 0 ? L.active : L.active2)) break;
    float *acc = acc_all + c * VN;
    if (a.self_term) {
      float v[VN];
      V::unpack(ld16<false>(reinterpret_cast<const char *>(sl.in) + ((size_t)r * sl.ldi + col) * V::BYTES, 0), v);
#pragma unroll
      for (int k = 0; k < VN; ++k) acc[k] = fmaf(ws, v[k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < VN; ++k) acc[k] *= sc;
    if (sl.axpy) {
      float v[VN];
      // coherent load: the axpy block may be the output block (in-place accumulate)
      V::unpack(ld16c<HINT>(reinterpret_cast<const char *>(sl.axpy) + ((size_t)r * sl.lda + col) * V::BYTES,
                            pol.stream),
                v);
#pragma unroll
      for (int k = 0; k < VN; ++k) acc[k] = fmaf(as, v[k], acc[k]);
    }
    for (int t = 0; t < a.lr_rank; ++t) {
      const int tu = t - a.lr_ones_first;
      const float u = (tu < 0 || !a.lr_u) ? 1.f : __ldg(a.lr_u + (size_t)r * a.lr_ldu + tu);
      const float al = a.lr_alpha[t] * u;
      const float *cf = a.lr_c + (size_t)t * a.lr_ldc + sl.col0 + col;
#pragma unroll
      for (int k = 0; k < VN; ++k) acc[k] = fmaf(al, __ldg(cf + k), acc[k]);
    }
    const int valid = min(VN, sl.width - col);
    char *o = reinterpret_cast<char *>(sl.out) + ((size_t)r * sl.ldo + col) * V::BYTES;
    if (valid >= VN) st16<HINT>(o, V::pack(acc), pol.stream);
    else V::store_partial(o, acc, valid);
  }
}

// L2 prefetch of the first neighbour rows of the group's next row: more
// requests in flight without holding registers.  Lane gl of the group takes
// nonzero gl / lines and 128-byte line gl % lines of its gathered row.
template <int DT>
__device__ __forceinline__ void prefetch_next_row(const SpmmArgs &a, const SpmmSlab &sl, const Lane &L, int64_t rn) {
  if (rn >= a.rows) return;
  const int e0 = __ldg(a.rowptr + rn), e1 = __ldg(a.rowptr + rn + 1);
  const int row_bytes = sl.width * Vec<DT>::BYTES;
  const int lines = (row_bytes + 127) / 128;
  const int t = L.gl / lines, line = L.gl - t * lines;
  if (e1 - e0 > a.heavy_threshold || t >= kPrefetchNonzeros || e0 + t >= e1 || line >= lines) return;
  const int32_t c = a.tagged ? (__ldg(a.tagged + e0 + t) & ((1 << 26) - 1)) : __ldg(a.colidx + e0 + t);
  const char *p = reinterpret_cast<const char *>(sl.in) + ((size_t)c * sl.ldi) * Vec<DT>::BYTES + line * 128;
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// GROUPED: some slab of the launch has several row groups per warp (the
// grouped gather is compiled in only then, so that one-group launches keep
// their registers).
template <int DT, bool HINT, int MINB, int CPL, bool GROUPED>
__global__ void __launch_bounds__(256, MINB) spmm_rows_kernel(const __grid_constant__ SpmmArgs a) {
  constexpr int VN = Vec<DT>::N;
  const SpmmSlab &sl = a.slab[blockIdx.y];
  const Lane L = make_lane<DT>(sl);
  const Policies pol = make_policies<HINT>();
  const int rpw = 32 / L.G;
  const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nwarp = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t base = warp * rpw; base < a.rows; base += nwarp * rpw) {
    const int64_t r = base + L.sub;
    if (!GROUPED || L.G == 32) {  // one row group per warp
      if (r >= a.rows) continue;
      const int e0 = ld_idx<HINT>(a.rowptr + r, pol.stream), e1 = ld_idx<HINT>(a.rowptr + r + 1, pol.stream);
      if (a.prefetch) prefetch_next_row<DT>(a, sl, L, r + nwarp * rpw);
      if (e1 - e0 > a.heavy_threshold) continue;  // heavy rows: chunks + finish
      float acc[CPL * VN];
#pragma unroll
      for (int k = 0; k < CPL * VN; ++k) acc[k] = 0.f;
      gather_range<DT, HINT, CPL>(a, sl, L, e0, e1, pol, acc);
      epilogue<DT, HINT, CPL>(a, sl, L, r, pol, acc);
    } else {
      // rows in degree order when there is one, so that a warp's groups have
      // rows of about the same length
      const bool in_range = r < a.rows;  // uniform within the group
      const int64_t rr = in_range && a.row_order ? (int64_t)__ldg(a.row_order + r) : r;
      int e0 = 0, e1 = 0;
      if (in_range) {
        e0 = ld_idx<HINT>(a.rowptr + rr, pol.stream);
        e1 = ld_idx<HINT>(a.rowptr + rr + 1, pol.stream);
        if (a.prefetch && !a.row_order) prefetch_next_row<DT>(a, sl, L, r + nwarp * rpw);
      }
      const bool mine = in_range && e1 - e0 <= a.heavy_threshold;
      const int len = mine ? e1 - e0 : 0;
      float acc[CPL * VN];
#pragma unroll
      for (int k = 0; k < CPL * VN; ++k) acc[k] = 0.f;
      gather_range_grouped<DT, HINT, CPL>(a, sl, L, e0, len, __reduce_max_sync(0xffffffffu, len), pol, acc);
      if (mine) epilogue<DT, HINT, CPL>(a, sl, L, rr, pol, acc);
    }
  }
}

template <int DT, bool HINT, int CPL, bool GROUPED>
__global__ void __launch_bounds__(256) spmm_chunks_kernel(const __grid_constant__ SpmmArgs a,
                                                          const int2 *__restrict__ chunks,
                                                          const int32_t *__restrict__ chunk_end, int32_t n,
                                                          float *__restrict__ partial, int64_t pw) {
  constexpr int VN = Vec<DT>::N;
  const SpmmSlab &sl = a.slab[blockIdx.y];
  const Lane L = make_lane<DT>(sl);
  const Policies pol = make_policies<HINT>();
  const int rpw = 32 / L.G;
  const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nwarp = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t base = warp * rpw; base < n; base += nwarp * rpw) {
    const int64_t c = base + L.sub;
    float acc[CPL * VN];
#pragma unroll
    for (int k = 0; k < CPL * VN; ++k) acc[k] = 0.f;
    if (!GROUPED || L.G == 32) {  // one chunk group per warp
      if (c >= n) continue;
      gather_range<DT, HINT, CPL>(a, sl, L, chunks[c].y, chunk_end[c], pol, acc);
    } else {
      const bool in_range = c < n;  // uniform within the group
      const int e0 = in_range ? chunks[c].y : 0, len = in_range ? chunk_end[c] - e0 : 0;
      gather_range_grouped<DT, HINT, CPL>(a, sl, L, e0, len, __reduce_max_sync(0xffffffffu, len), pol, acc);
      if (!in_range) continue;
    }
#pragma unroll
    for (int h = 0; h < CPL; ++h) {
      if (!(h == 0 ? L.active : L.active2)) break;
      float *p = partial + (size_t)c * pw + sl.col0 + (h == 0 ? L.col : L.col2);
#pragma unroll
      for (int k = 0; k < VN; ++k) p[k] = acc[h * VN + k];
    }
  }
}

template <int DT, bool HINT, int CPL>
__global__ void __launch_bounds__(256) spmm_finish_kernel(const __grid_constant__ SpmmArgs a,
                                                          const int4 *__restrict__ hrows, int32_t n,
                                                          const float *__restrict__ partial, int64_t pw) {
  constexpr int VN = Vec<DT>::N;
  const SpmmSlab &sl = a.slab[blockIdx.y];
  const Lane L = make_lane<DT>(sl);
  const Policies pol = make_policies<HINT>();
  const int rpw = 32 / L.G;
  const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nwarp = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t base = warp * rpw; base < n; base += nwarp * rpw) {
    const int64_t h = base + L.sub;
    if (h >= n) continue;
    const int4 hr = hrows[h];
    float acc[CPL * VN];
#pragma unroll
    for (int k = 0; k < CPL * VN; ++k) acc[k] = 0.f;
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      if (!(q == 0 ? L.active : L.active2)) break;
      // chunk partials in order, 8 loads in flight (the largest hubs have hundreds)
      const float *p0 = partial + (size_t)hr.y * pw + sl.col0 + (q == 0 ? L.col : L.col2);
      int c = 0;
      constexpr int NV = VN / 4;  // float4 per lane and chunk
      for (; c + 8 <= hr.z; c += 8) {
        float4 v[8][NV];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int h = 0; h < NV; ++h)
            v[u][h] = __ldcg(reinterpret_cast<const float4 *>(p0 + (size_t)(c + u) * pw) + h);
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int h = 0; h < NV; ++h) {
            acc[q * VN + 4 * h + 0] += v[u][h].x;
            acc[q * VN + 4 * h + 1] += v[u][h].y;
            acc[q * VN + 4 * h + 2] += v[u][h].z;
            acc[q * VN + 4 * h + 3] += v[u][h].w;
          }
      }
      for (; c < hr.z; ++c) {
        const float *p = p0 + (size_t)c * pw;
#pragma unroll
        for (int k = 0; k < VN; ++k) acc[q * VN + k] += p[k];
      }
    }
    epilogue<DT, HINT, CPL>(a, sl, L, hr.x, pol, acc);
  }
}

// Rows with many chunks (the first n_big of the plan): one CTA per row and
// slab; warp w sums chunks w, w + 8, ... (in order), the eight warp sums are
// added in warp order, and warp 0 applies the epilogue.  Lanes past the first
// row group of a warp (narrow slabs) stay idle.
template <int DT, bool HINT, int CPL>
__global__ void __launch_bounds__(256) spmm_finish_big_kernel(const __grid_constant__ SpmmArgs a,
                                                              const int4 *__restrict__ hrows,
                                                              const float *__restrict__ partial, int64_t pw) {
  constexpr int VN = Vec<DT>::N;
  constexpr int NW = 8;
  __shared__ float4 red[NW][32][CPL * VN / 4];
  const SpmmSlab &sl = a.slab[blockIdx.y];
  const Lane L = make_lane<DT>(sl);
  const Policies pol = make_policies<HINT>();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int4 hr = hrows[blockIdx.x];
  float acc[CPL * VN];
#pragma unroll
  for (int k = 0; k < CPL * VN; ++k) acc[k] = 0.f;
  if (L.sub == 0) {
    constexpr int NV = VN / 4;  // float4 per lane and chunk
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
      if (!(q == 0 ? L.active : L.active2)) break;
      const float *p0 = partial + (size_t)hr.y * pw + sl.col0 + (q == 0 ? L.col : L.col2);
      int c = warp;
      for (; c + 3 * NW < hr.z; c += 4 * NW) {
        float4 v[4][NV];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int h = 0; h < NV; ++h)
            v[u][h] = __ldcg(reinterpret_cast<const float4 *>(p0 + (size_t)(c + u * NW) * pw) + h);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int h = 0; h < NV; ++h) {
            acc[q * VN + 4 * h + 0] += v[u][h].x;
            acc[q * VN + 4 * h + 1] += v[u][h].y;
            acc[q * VN + 4 * h + 2] += v[u][h].z;
            acc[q * VN + 4 * h + 3] += v[u][h].w;
          }
      }
      for (; c < hr.z; c += NW) {
        const float *pc = p0 + (size_t)c * pw;
#pragma unroll
        for (int k = 0; k < VN; ++k) acc[q * VN + k] += pc[k];
      }
    }
  }
#pragma unroll
  for (int k = 0; k < CPL * VN / 4; ++k)
    red[warp][lane][k] = make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
  __syncthreads();
  if (warp == 0 && L.sub == 0) {
#pragma unroll
    for (int k = 0; k < CPL * VN / 4; ++k) {
      float4 t = red[0][lane][k];
#pragma unroll
      for (int w = 1; w < NW; ++w) {
        const float4 u = red[w][lane][k];
        t.x += u.x;
        t.y += u.y;
        t.z += u.z;
        t.w += u.w;
      }
      acc[4 * k] = t.x;
      acc[4 * k + 1] = t.y;
      acc[4 * k + 2] = t.z;
      acc[4 * k + 3] = t.w;
    }
    epilogue<DT, HINT, CPL>(a, sl, L, hr.x, pol, acc);
  }
}

// Packed-slab gather: acc += sum over the segment [e0, e0 + len) of
// a_e w_j in_j for the lane's 16-byte chunk of the slab.  The groups of a
// warp step together to the warp's longest segment (maxlen); every lane of
// the warp calls it.  The segment is taken 32 nonzeros at a time (4 G for
// groups of fewer than eight lanes): the G lanes of a group first load all the
// block's column indices (one coalesced load per index and lane), then
// issue its gathers four at a time, so that a row costs one index round trip
// per block whatever the slab width.
template <int DT, int G, bool WEIGHTED, bool HINT>
__device__ __forceinline__ void gather_segment(const SpmmArgs &a, const SpmmSlab &sl, const Lane &L, int e0,
                                               int len, int maxlen, const Policies &pol, float *acc) {
  using V = Vec<DT>;
  constexpr int VN = V::N;
  constexpr int U = G < 4 ? G : 4;
  constexpr int IPL = G >= 8 ? 32 / G : 4;  // indices per lane and block
  constexpr int BLK = IPL * G;              // nonzeros per block (32, or 4 G for the narrowest groups)
  const char *inb = reinterpret_cast<const char *>(sl.in) + (size_t)L.col * V::BYTES;
  const size_t ldb = (size_t)sl.ldi * V::BYTES;
  const int lead = L.sub * G;
  const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
  for (int off = 0; off < maxlen; off += BLK) {
    int j[IPL];
    float w[WEIGHTED ? IPL : 1];
#pragma unroll
    for (int q = 0; q < IPL; ++q) {
      const int t = off + q * G + L.gl;
      j[q] = -1;
      if (WEIGHTED) w[q] = 1.f;
      if (t < len) {
        const int e = e0 + t;
        j[q] = ld_idx<HINT>(a.colidx + e, pol.stream);
        if (WEIGHTED) {
          w[q] = a.values ? __ldg(a.values + e) : 1.f;
          if (a.colw) w[q] *= __ldg(a.colw + j[q]);
        }
      }
    }
    const int cnt = min(BLK, maxlen - off);  // warp-uniform
#pragma unroll
    for (int q = 0; q < IPL; ++q) {
      if (q * G >= cnt) break;
#pragma unroll
      for (int u0 = 0; u0 < G; u0 += U) {
        int jj[U];
        float ww[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          jj[u] = __shfl_sync(0xffffffffu, j[q], lead + u0 + u);
          ww[u] = WEIGHTED ? __shfl_sync(0xffffffffu, w[WEIGHTED ? q : 0], lead + u0 + u) : 1.f;
        }
        if (L.active) {
          uint4 raw[U];
#pragma unroll
          for (int u = 0; u < U; ++u)
            raw[u] = jj[u] >= 0 ? ld16<HINT && ISVD_SLAB_GATHER_KEEP>(inb + (size_t)jj[u] * ldb, pol.keep) : zero;
#pragma unroll
          for (int u = 0; u < U; ++u) {
            float v[VN];
            V::unpack(raw[u], v);
#pragma unroll
            for (int k = 0; k < VN; ++k) acc[k] = fmaf(ww[u], v[k], acc[k]);
          }
        }
      }
    }
  }
}

// One column slab (a.slab[0]) over the packed-slab work list: `group` lanes
// per segment, 32 / group segments per warp.  Whole rows end in the epilogue;
// hub pieces store partials, and the group that finishes a hub's last piece
// sums the hub's partials in slot order and runs the epilogue.
template <int DT, int G, int MINB, bool HINT>
__global__ void __launch_bounds__(256, MINB)
    spmm_slab_kernel(const __grid_constant__ SpmmArgs a, const int4 *__restrict__ items, int32_t n_items,
                     const int4 *__restrict__ hubs, const int32_t *__restrict__ slot_hub, int32_t *counters,
                     float *partial, int64_t pw) {
  constexpr int VN = Vec<DT>::N;
  const SpmmSlab &sl = a.slab[0];
  const Lane L = make_lane<DT>(sl);  // sl.group == G
  Policies pol{0, 0};
  if (HINT) pol = Policies{policy_keep(), policy_stream()};
  constexpr int rpw = 32 / G;
  const bool weighted = a.values != nullptr || a.colw != nullptr;
  const int64_t warp = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t nwarp = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t base = warp * rpw; base < n_items; base += nwarp * rpw) {
    const int64_t it = base + L.sub;
    int4 item = make_int4(0, 0, 0, -2);  // slot -2: no segment for this group
    if (it < n_items) item = __ldg(items + it);
    const int len = item.z - item.y;
    const int maxlen = __reduce_max_sync(0xffffffffu, len);
    float acc[VN];
#pragma unroll
    for (int k = 0; k < VN; ++k) acc[k] = 0.f;
    if (weighted) gather_segment<DT, G, true, HINT>(a, sl, L, item.y, len, maxlen, pol, acc);
    else gather_segment<DT, G, false, HINT>(a, sl, L, item.y, len, maxlen, pol, acc);
    if (item.w == -2) continue;
    if (item.w == -1) {
      epilogue<DT, HINT, 1>(a, sl, L, item.x, pol, acc);
      continue;
    }
    // a hub piece: publish the partial, then count it
    if (L.active) {
      float4 *p = reinterpret_cast<float4 *>(partial + (size_t)item.w * pw + L.col);
#pragma unroll
      for (int k = 0; k < VN / 4; ++k) p[k] = make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
    }
    __threadfence();
    __syncwarp(L.mask);
    const int h = __ldg(slot_hub + item.w);
    int done = 0;
    if (L.gl == 0) done = atomicAdd(counters + h, 1) + 1;
    done = __shfl_sync(L.mask, done, L.sub * L.G);
    const int4 hb = __ldg(hubs + h);
    if (done != hb.z) continue;
    // last piece of the hub: every other piece's partial is visible (fence before each count)
    __threadfence();
#pragma unroll
    for (int k = 0; k < VN; ++k) acc[k] = 0.f;
    if (L.active) {
      for (int c = 0; c < hb.z; ++c) {
        const float4 *q = reinterpret_cast<const float4 *>(partial + (size_t)(hb.y + c) * pw + L.col);
#pragma unroll
        for (int k = 0; k < VN / 4; ++k) {
          const float4 v = __ldcg(q + k);
          acc[4 * k] += v.x;
          acc[4 * k + 1] += v.y;
          acc[4 * k + 2] += v.z;
          acc[4 * k + 3] += v.w;
        }
      }
    }
    epilogue<DT, HINT, 1>(a, sl, L, hb.x, pol, acc);
    if (L.gl == 0) counters[h] = 0;  // ready for the next launch
  }
}

int pow2_ceil(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

template <int DT, bool HINT, int CPL>
cudaError_t launch_cpl(const SpmmArgs &a, const HeavyPlan &hp, float *partial, int64_t pw, cudaStream_t s,
                       const SideStream &side) {
  const int threads = 256;
  int gmin = 32;
  for (int i = 0; i < a.nslabs; ++i) gmin = gmin < a.slab[i].group ? gmin : a.slab[i].group;
  const bool grouped = gmin < 32;
  const int64_t rows_per_block = (threads / 32) * (32 / gmin);
  int64_t bx = ceil_div(a.rows, rows_per_block);
  const int64_t cap = (int64_t)kNumSMs * 16;
  if (bx > cap) bx = cap;
  if (bx < 1) bx = 1;
  dim3 grid((unsigned)bx, (unsigned)a.nslabs);
  // the hub chunks (their own partial buffer, no row in common with the row
  // kernel) run on the side stream when there is one, filling the row kernel's tail
  const bool fork = hp.n_chunks > 0 && side.stream && side.fork && side.join;
  cudaStream_t hs = fork ? side.stream : s;
  if (fork) {
    cudaError_t e = cudaEventRecord(side.fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side.stream, side.fork, 0);
    if (e != cudaSuccess) return e;
  }
  if (hp.n_chunks > 0) {
    int64_t cx = ceil_div(hp.n_chunks, rows_per_block);
    if (cx > cap) cx = cap;
    if (grouped)
      spmm_chunks_kernel<DT, HINT, CPL, true><<<dim3((unsigned)cx, (unsigned)a.nslabs), threads, 0, hs>>>(
          a, hp.chunks, hp.chunk_end, hp.n_chunks, partial, pw);
    else
      spmm_chunks_kernel<DT, HINT, CPL, false><<<dim3((unsigned)cx, (unsigned)a.nslabs), threads, 0, hs>>>(
          a, hp.chunks, hp.chunk_end, hp.n_chunks, partial, pw);
  }
  // high occupancy: 6 blocks of 256 threads per SM (40 registers) for FP32;
  // BF16 rows hold twice the accumulators and take 5 (48 registers, no spills)
  constexpr int kHighOcc = CPL == 2 ? ISVD_WIDE_MINB : DT == DT_F32 ? ISVD_ROWS_HIGH_OCC_F32 : 5;
  if (a.rows_occupancy >= 3 && grouped)
    spmm_rows_kernel<DT, HINT, kHighOcc, CPL, true><<<grid, threads, 0, s>>>(a);
  else if (a.rows_occupancy >= 3)
    spmm_rows_kernel<DT, HINT, kHighOcc, CPL, false><<<grid, threads, 0, s>>>(a);
  else if (grouped)
    spmm_rows_kernel<DT, HINT, 1, CPL, true><<<grid, threads, 0, s>>>(a);
  else
    spmm_rows_kernel<DT, HINT, 1, CPL, false><<<grid, threads, 0, s>>>(a);
  if (fork) {
    cudaError_t e = cudaEventRecord(side.join, side.stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, side.join, 0);
    if (e != cudaSuccess) return e;
  }
  if (hp.n_big > 0)
    spmm_finish_big_kernel<DT, HINT, CPL><<<dim3((unsigned)hp.n_big, (unsigned)a.nslabs), threads, 0, s>>>(
        a, hp.rows, partial, pw);
  if (hp.n_rows > hp.n_big) {
    int64_t fx = ceil_div(hp.n_rows - hp.n_big, rows_per_block);
    if (fx > cap) fx = cap;
    spmm_finish_kernel<DT, HINT, CPL><<<dim3((unsigned)fx, (unsigned)a.nslabs), threads, 0, s>>>(
        a, hp.rows + hp.n_big, hp.n_rows - hp.n_big, partial, pw);
  }
  return cudaGetLastError();
}

// Wide slabs (more than 32 chunks of 16 bytes) use two chunks per lane.
template <int DT, bool HINT>
cudaError_t launch_dt(const SpmmArgs &a, const HeavyPlan &hp, float *partial, int64_t pw, cudaStream_t s,
                      const SideStream &side) {
  bool wide = false;
  for (int i = 0; i < a.nslabs; ++i) wide = wide || a.slab[i].width > a.slab[i].group * Vec<DT>::N;
  return wide ? launch_cpl<DT, HINT, 2>(a, hp, partial, pw, s, side)
              : launch_cpl<DT, HINT, 1>(a, hp, partial, pw, s, side);
}

}  // namespace

// Slabs of at most slab_cols columns.  Up to 32 * vn columns a slab gives each
// lane of its row group one 16-byte chunk; wider slab_cols (wide mode) give
// each lane two chunks when a slab has more than 16, so that rows of 17..64
// chunks pack into groups of half the lanes (e.g. 144 BF16 columns: 2 rows
// per warp instead of 1 with 14 idle lanes).
int make_slabs(int dtype, int32_t b, int32_t slab_cols, SpmmSlab *out) {
  const int vn = dtype == DT_F32 ? 4 : 8;
  const bool wide = slab_cols > 32 * vn;
  int max_cols = 64 * vn;  // 32 lanes x two 16-byte chunks
  if (slab_cols > max_cols) slab_cols = max_cols;
  if (slab_cols < vn) slab_cols = vn;
  int n = 0;
  for (int c0 = 0; c0 < b; c0 += slab_cols) {
    const int w = (b - c0) < slab_cols ? (b - c0) : slab_cols;
    SpmmSlab sl{};
    sl.col0 = c0;
    sl.width = w;
    const int chunks = (w + vn - 1) / vn;
    sl.group = (wide && chunks > 16) ? pow2_ceil((chunks + 1) / 2) : pow2_ceil(chunks);
    out[n++] = sl;
  }
  return n;
}

constexpr bool kSlabHints = true;

template <int DT, int MINB>
cudaError_t slab_launch_one(const SpmmArgs &one, const SlabPlan &p, float *partial, int64_t pw, cudaStream_t s) {
  const int G = one.slab[0].group;
  int64_t bx = ceil_div(p.n_items, 8 * (32 / G));
  const int64_t cap = (int64_t)kNumSMs * MINB;
  if (bx > cap) bx = cap;
  const dim3 grid((unsigned)bx);
#define ISVD_SLAB_CASE(g)                                                                                      \
  case g:                                                                                                      \
    spmm_slab_kernel<DT, g, MINB, kSlabHints><<<grid, 256, 0, s>>>(one, p.items, p.n_items, p.hubs, p.slot_hub,  \
                                                                   p.counters, partial, pw);                   \
    break;
  switch (G) {
    ISVD_SLAB_CASE(1)
    ISVD_SLAB_CASE(2)
    ISVD_SLAB_CASE(4)
    ISVD_SLAB_CASE(8)
    ISVD_SLAB_CASE(16)
    ISVD_SLAB_CASE(32)
    default:
      return cudaErrorInvalidValue;
  }
#undef ISVD_SLAB_CASE
  return cudaGetLastError();
}

cudaError_t spmm_slab_launch(const SpmmArgs &a, int dtype, const SlabPlan &p, float *partial, int64_t pw,
                             cudaStream_t s) {
  if (a.rows == 0 || a.nslabs == 0 || p.n_items == 0) return cudaSuccess;
  for (int i = 0; i < a.nslabs; ++i) {
    SpmmArgs one = a;
    one.slab[0] = a.slab[i];
    one.nslabs = 1;
    const cudaError_t e = dtype == DT_F32 ? slab_launch_one<DT_F32, ISVD_SLAB_MINB_F32>(one, p, partial, pw, s)
                                          : slab_launch_one<DT_BF16, ISVD_SLAB_MINB_BF16>(one, p, partial, pw, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t spmm_launch(const SpmmArgs &a, int dtype, const HeavyPlan &hp, float *partial, int64_t pw,
                        cudaStream_t s, const SideStream &side) {
  if (a.rows == 0 || a.nslabs == 0) return cudaSuccess;
  if (a.cache_hints)
    return dtype == DT_F32 ? launch_dt<DT_F32, true>(a, hp, partial, pw, s, side)
                           : launch_dt<DT_BF16, true>(a, hp, partial, pw, s, side);
  return dtype == DT_F32 ? launch_dt<DT_F32, false>(a, hp, partial, pw, s, side)
                         : launch_dt<DT_BF16, false>(a, hp, partial, pw, s, side);
}

}  // namespace isvd
