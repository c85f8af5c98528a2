// The implicit operator: construction (validation, degrees, scale vectors,
// X^T, row work lists) and the products M.G / M^T.G (Sec. 4, App. A.3).
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <string>

#include <atomic>

#include "internal.h"

namespace isvd {

static thread_local std::string g_last_error;

void set_error(const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

isvd_status fail(isvd_status s, const char *fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

const char *last_error() { return g_last_error.c_str(); }

void *op_alloc(isvd_operator *op, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  bytes = (size_t)round_up((int64_t)bytes, 256);
  if (op->has_alloc) return op->alloc.alloc(bytes, (void *)s, op->alloc.ctx);
  void *p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void op_free(isvd_operator *op, void *p, cudaStream_t s) {
  if (!p) return;
  if (op->has_alloc) op->alloc.free(p, (void *)s, op->alloc.ctx);
  else cudaFreeAsync(p, s);
}

void invalidate_graphs(isvd_operator *op) {
  for (auto &g : op->graphs) cudaGraphExecDestroy(g.exec);
  op->graphs.clear();
  ++op->generation;
}

isvd_status ensure_arena(isvd_operator *op, size_t bytes, cudaStream_t s) {
  if (bytes <= op->arena_bytes) return ISVD_OK;
  invalidate_graphs(op);  // captured graphs point into the old arena
  op_free(op, op->arena, s);
  op->arena = nullptr;
  op->arena_bytes = 0;
  const size_t want = (size_t)round_up((int64_t)bytes, 1 << 20);
  op->arena = op_alloc(op, want, s);
  if (!op->arena) return fail(ISVD_ERR_WORKSPACE, "workspace allocation of %zu bytes failed", want);
  op->arena_bytes = want;
  return ISVD_OK;
}

namespace {

// ---- construction kernels ----------------------------------------------------
// flags: [0] rowptr malformed  [1] column index out of range  [2] non-finite value
//        [3] zero or negative degree where T = D^-1 A needs 1/d
// Row gather indices: in [0, rows) and strictly increasing; flags[0] = 1 otherwise.
__global__ void validate_rows_kernel(const int32_t *idx, int64_t count, int64_t rows, int32_t *flags) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const int32_t r = idx[i];
    if (r < 0 || r >= rows || (i > 0 && idx[i - 1] >= r)) flags[0] = 1;
  }
}

// out[i][:b] = full[idx[i]][:b] (gather) or full[idx[i]][:b] = in[i][:b]
// (scatter into a zeroed block), element type T.
template <typename T>
__global__ void gather_rows_kernel(const T *src, int64_t lds, const int32_t *idx, int64_t count, int32_t b, T *dst,
                                   int64_t ldd, int32_t scatter) {
  const int64_t total = count * b;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t i = e / b, c = e - i * b;
    const int64_t r = idx[i];
    if (scatter) dst[r * ldd + c] = src[i * lds + c];
    else dst[i * ldd + c] = src[r * lds + c];
  }
}

__device__ __forceinline__ float blk_load(const float *p) { return *p; }
__device__ __forceinline__ float blk_load(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ void blk_store(float *p, float v) { *p = v; }
__device__ __forceinline__ void blk_store(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// y = w x (first) or y + w x over a rows x b block, in FP32 (x may be y).
template <typename T>
__global__ void axpy_block_kernel(const T *x, int64_t ldx, T *y, int64_t ldy, int64_t rows, int32_t b, float w,
                                  int32_t first) {
  const int64_t total = rows * b;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t i = e / b, c = e - i * b;
    const float xv = w * blk_load(x + i * ldx + c);
    T *py = y + i * ldy + c;
    blk_store(py, first ? xv : blk_load(py) + xv);
  }
}

__global__ void validate_csr_kernel(int64_t rows, int64_t cols, int64_t nnz, const int32_t *rowptr,
                                    const int32_t *colidx, const float *values, int32_t *flags) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= rows; i += stride) {
    const int32_t a = rowptr[i];
    if (i == 0 && a != 0) flags[0] = 1;
    if (i == rows && (int64_t)a != nnz) flags[0] = 1;
    if (i < rows && rowptr[i + 1] < a) flags[0] = 1;
  }
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
    const int32_t c = colidx[e];
    if (c < 0 || (int64_t)c >= cols) flags[1] = 1;
    if (values && !isfinite(values[e])) flags[2] = 1;
  }
}

// d_i = sum_j A_ij (Sec. 2); 1/d_i for T = D^-1 A; s_i = (d_i + 1)^-1/2 and
// s_i^2 for Â = (D+I)^-1/2 (A+I) (D+I)^-1/2.
__global__ void degree_kernel(int64_t n, const int32_t *rowptr, const float *values, int need_positive, float *deg,
                              float *inv_d, float *s, float *s2, int32_t *flags) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int32_t e0 = rowptr[i], e1 = rowptr[i + 1];
    double d = 0.0;
    if (values) {
      for (int32_t e = e0; e < e1; ++e) d += (double)values[e];
    } else {
      d = (double)(e1 - e0);
    }
    deg[i] = (float)d;
    if (need_positive && !(d > 0.0)) flags[3] = 1;
    inv_d[i] = d > 0.0 ? (float)(1.0 / d) : 0.f;
    if (d + 1.0 <= 0.0) flags[3] = 1;
    const double si = d + 1.0 > 0.0 ? 1.0 / sqrt(d + 1.0) : 0.0;
    s[i] = (float)si;
    s2[i] = (float)(si * si);
  }
}

__global__ void edge_keys_kernel(int64_t n, int64_t nnz, const int32_t *rowptr, const int32_t *colidx,
                                 uint64_t *key_rc, uint64_t *key_cr) {
  // one thread per row (rows are short on average); keys (row, col) and (col, row)
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const uint64_t c = (uint64_t)colidx[e];
      key_rc[e] = (uint64_t)i * (uint64_t)n + c;
      key_cr[e] = c * (uint64_t)n + (uint64_t)i;
    }
  }
}

__global__ void compare_kernel(int64_t nnz, const uint64_t *ka, const uint64_t *kb, const float *va,
                               const float *vb, int32_t *flags) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
    if (ka[e] != kb[e]) flags[4] = 1;
    if (va && va[e] != vb[e]) flags[4] = 1;
  }
}

__global__ void iota_kernel(int64_t n, int32_t *out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (int32_t)i;
}

__global__ void row_of_entry_kernel(int64_t rows, const int32_t *rowptr, int32_t *row_of) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += stride)
    for (int32_t e = rowptr[i]; e < rowptr[i + 1]; ++e) row_of[e] = (int32_t)i;
}

__global__ void gather_transpose_kernel(int64_t nnz, const int32_t *perm, const int32_t *row_of,
                                        const float *values, int32_t *t_colidx, float *t_values) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride) {
    const int32_t e = perm[p];
    t_colidx[p] = row_of[e];
    t_values[p] = values ? values[e] : 1.f;
  }
}

__global__ void count_kernel(int64_t nnz, const int32_t *keys, int32_t *counts) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride)
    atomicAdd(&counts[keys[e]], 1);
}

__global__ void dense_csr_kernel(int64_t n, int64_t d, int32_t *rowptr, int32_t *colidx) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) rowptr[i] = (int32_t)(i * d);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * d; e += stride)
    colidx[e] = (int32_t)(e % d);
}

unsigned grid_for(int64_t work) {
  int64_t b = ceil_div(work, 256);
  if (b > kNumSMs * 8) b = kNumSMs * 8;
  if (b < 1) b = 1;
  return (unsigned)b;
}

int bits_for(uint64_t maxval) {
  int b = 1;
  while (b < 64 && (maxval >> b) != 0) ++b;
  return b;
}

struct Scratch {
  isvd_operator *op;
  cudaStream_t s;
  std::vector<void *> ptrs;
  void *get(size_t bytes) {
    void *p = op_alloc(op, bytes, s);
    if (p) ptrs.push_back(p);
    return p;
  }
  ~Scratch() {
    for (void *p : ptrs) op_free(op, p, s);
  }
};

void *owned_alloc(isvd_operator *op, size_t bytes, cudaStream_t s) {
  void *p = op_alloc(op, bytes, s);
  if (p) op->owned.push_back(p);
  return p;
}

}  // namespace

void free_heavy(isvd_operator *op, HeavyPlan *hp, cudaStream_t s) {
  op_free(op, hp->chunks, s);
  op_free(op, hp->chunk_end, s);
  op_free(op, hp->rows, s);
  hp->chunks = nullptr;
  hp->chunk_end = nullptr;
  hp->rows = nullptr;
  hp->n_rows = hp->n_chunks = hp->n_big = 0;
}

void free_chunks(isvd_operator *op, ChunkPlan *cp, cudaStream_t s) {
  op_free(op, cp->row_of, s);
  op_free(op, cp->split, s);
  op_free(op, cp->empty, s);
  cp->row_of = nullptr;
  cp->split = nullptr;
  cp->empty = nullptr;
  cp->nchunks = cp->nsplit = cp->nempty = 0;
}

void free_slab_plan(isvd_operator *op, SlabPlan *sp, cudaStream_t s) {
  op_free(op, sp->items, s);
  op_free(op, sp->hubs, s);
  op_free(op, sp->slot_hub, s);
  op_free(op, sp->counters, s);
  sp->items = nullptr;
  sp->hubs = nullptr;
  sp->slot_hub = nullptr;
  sp->counters = nullptr;
  sp->n_items = sp->n_hubs = sp->n_slots = 0;
}

namespace {

// Packed-slab work list from a host copy of rowptr: whole rows of at most
// `threshold` nonzeros and `chunk`-nonzero pieces of the longer rows, sorted by
// length, longest first (ties in row order), so that the groups of a warp get
// segments of about the same length.
isvd_status build_slab_plan(isvd_operator *op, const int32_t *rowptr_dev, int64_t rows, int32_t threshold,
                            int32_t chunk, SlabPlan *sp, cudaStream_t s) {
  std::vector<int32_t> rp((size_t)rows + 1);
  ISVD_CUDA_TRY(cudaMemcpyAsync(rp.data(), rowptr_dev, sizeof(int32_t) * (rows + 1), cudaMemcpyDeviceToHost, s));
  ISVD_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int4> items;
  std::vector<int4> hubs;
  std::vector<int32_t> slot_hub;
  items.reserve((size_t)rows);
  for (int64_t i = 0; i < rows; ++i) {
    const int32_t e0 = rp[i], e1 = rp[i + 1];
    if (e1 - e0 <= threshold) {
      items.push_back(make_int4((int)i, e0, e1, -1));
      continue;
    }
    const int32_t first = (int32_t)slot_hub.size();
    for (int32_t e = e0; e < e1; e += chunk) {
      items.push_back(make_int4((int)i, e, std::min<int32_t>(e1, e + chunk), (int)slot_hub.size()));
      slot_hub.push_back((int32_t)hubs.size());
    }
    hubs.push_back(make_int4((int)i, first, (int32_t)slot_hub.size() - first, 0));
  }
  // counting sort by length, longest first, stable
  const int32_t maxlen = std::max(threshold, chunk);
  std::vector<int64_t> pos((size_t)maxlen + 2, 0);
  for (const int4 &t : items) pos[t.z - t.y] += 1;
  int64_t acc = 0;
  for (int64_t len = maxlen; len >= 0; --len) {
    const int64_t c = pos[len];
    pos[len] = acc;
    acc += c;
  }
  std::vector<int4> sorted(items.size());
  for (const int4 &t : items) sorted[pos[t.z - t.y]++] = t;
  free_slab_plan(op, sp, s);
  sp->chunk = chunk;
  sp->n_items = (int32_t)sorted.size();
  sp->n_hubs = (int32_t)hubs.size();
  sp->n_slots = (int32_t)slot_hub.size();
  if (sp->n_items == 0) return ISVD_OK;
  sp->items = (int4 *)op_alloc(op, sizeof(int4) * sorted.size(), s);
  if (!sp->items) return fail(ISVD_ERR_WORKSPACE, "slab work list allocation failed");
  ISVD_CUDA_TRY(cudaMemcpyAsync(sp->items, sorted.data(), sizeof(int4) * sorted.size(), cudaMemcpyHostToDevice, s));
  if (sp->n_hubs > 0) {
    sp->hubs = (int4 *)op_alloc(op, sizeof(int4) * hubs.size(), s);
    sp->slot_hub = (int32_t *)op_alloc(op, sizeof(int32_t) * slot_hub.size(), s);
    sp->counters = (int32_t *)op_alloc(op, sizeof(int32_t) * hubs.size(), s);
    if (!sp->hubs || !sp->slot_hub || !sp->counters) return fail(ISVD_ERR_WORKSPACE, "slab hub plan allocation failed");
    ISVD_CUDA_TRY(cudaMemcpyAsync(sp->hubs, hubs.data(), sizeof(int4) * hubs.size(), cudaMemcpyHostToDevice, s));
    ISVD_CUDA_TRY(
        cudaMemcpyAsync(sp->slot_hub, slot_hub.data(), sizeof(int32_t) * slot_hub.size(), cudaMemcpyHostToDevice, s));
    ISVD_CUDA_TRY(cudaMemsetAsync(sp->counters, 0, sizeof(int32_t) * hubs.size(), s));
  }
  ISVD_CUDA_TRY(cudaStreamSynchronize(s));
  return ISVD_OK;
}

// Build the hub-row split plan from a host copy of rowptr.
isvd_status build_heavy(isvd_operator *op, const int32_t *rowptr_dev, int64_t rows, HeavyPlan *hp,
                        cudaStream_t s) {
  std::vector<int32_t> rp((size_t)rows + 1);
  ISVD_CUDA_TRY(cudaMemcpyAsync(rp.data(), rowptr_dev, sizeof(int32_t) * (rows + 1), cudaMemcpyDeviceToHost, s));
  ISVD_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int2> chunks;
  std::vector<int32_t> ends;
  std::vector<int4> hrows;
  for (int64_t i = 0; i < rows; ++i) {
    const int32_t e0 = rp[i], e1 = rp[i + 1];
    if (e1 - e0 <= hp->threshold) continue;
    const int first = (int)chunks.size();
    for (int32_t e = e0; e < e1; e += hp->chunk) {
      chunks.push_back(make_int2((int)i, e));
      ends.push_back(std::min<int32_t>(e1, e + hp->chunk));
    }
    hrows.push_back(make_int4((int)i, first, (int)chunks.size() - first, 0));
  }
  // rows by chunk count, most first (ties in row order): the rows with more than
  // kBigHubChunks chunks form a prefix (a whole CTA each), and the row groups of a
  // warp in the finish of the rest get about the same number of chunks
  std::stable_sort(hrows.begin(), hrows.end(), [](const int4 &x, const int4 &y) { return x.z > y.z; });
  int32_t n_big = 0;
  for (const int4 &h : hrows) n_big += h.z > kBigHubChunks ? 1 : 0;
  free_heavy(op, hp, s);
  hp->n_big = n_big;
  hp->n_rows = (int32_t)hrows.size();
  hp->n_chunks = (int32_t)chunks.size();
  if (hp->n_chunks == 0) return ISVD_OK;
  hp->chunks = (int2 *)op_alloc(op, sizeof(int2) * chunks.size(), s);
  hp->chunk_end = (int32_t *)op_alloc(op, sizeof(int32_t) * ends.size(), s);
  hp->rows = (int4 *)op_alloc(op, sizeof(int4) * hrows.size(), s);
  if (!hp->chunks || !hp->chunk_end || !hp->rows) return fail(ISVD_ERR_WORKSPACE, "heavy-row plan allocation failed");
  ISVD_CUDA_TRY(cudaMemcpyAsync(hp->chunks, chunks.data(), sizeof(int2) * chunks.size(), cudaMemcpyHostToDevice, s));
  ISVD_CUDA_TRY(cudaMemcpyAsync(hp->chunk_end, ends.data(), sizeof(int32_t) * ends.size(), cudaMemcpyHostToDevice, s));
  ISVD_CUDA_TRY(cudaMemcpyAsync(hp->rows, hrows.data(), sizeof(int4) * hrows.size(), cudaMemcpyHostToDevice, s));
  ISVD_CUDA_TRY(cudaStreamSynchronize(s));
  return ISVD_OK;
}

// Column tags for the ring form: colidx with floor(log2 deg_j) of the column's
// row degree in bits 26..30 (a column is re-read once per nonzero of it, so
// for symmetric A its degree is how often its row of the block is gathered).
__global__ void tag_columns_kernel(int64_t nnz, const int32_t *colidx, const int32_t *rowptr, int32_t *tagged) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
    const int32_t j = colidx[e];
    const int32_t d = rowptr[j + 1] - rowptr[j];
    const int32_t b = d > 0 ? 31 - __clz(d) : 0;
    tagged[e] = j | (b << 26);
  }
}

isvd_status build_tags(isvd_operator *op, cudaStream_t s) {
  const isvd_csr &A = op->desc.A;
  op->tags_A = RingTags{};
  if (op->n >= ((int64_t)1 << 26) || A.nnz == 0) return ISVD_OK;
  std::vector<int32_t> rp((size_t)op->n + 1);
  ISVD_CUDA_TRY(cudaMemcpyAsync(rp.data(), A.rowptr, sizeof(int32_t) * (op->n + 1), cudaMemcpyDeviceToHost, s));
  ISVD_CUDA_TRY(cudaStreamSynchronize(s));
  int32_t *t = (int32_t *)owned_alloc(op, sizeof(int32_t) * A.nnz, s);
  if (!t) return fail(ISVD_ERR_WORKSPACE, "column tag allocation failed");
  tag_columns_kernel<<<grid_for(A.nnz), 256, 0, s>>>(A.nnz, A.colidx, A.rowptr, t);
  ISVD_CUDA_TRY(cudaGetLastError());
  for (int64_t i = 0; i < op->n; ++i) {
    const int32_t d = rp[i + 1] - rp[i];
    int b = 0;
    while (b < 31 && (d >> (b + 1)) > 0) ++b;
    op->tags_A.hist[d > 0 ? b : 0] += 1;
  }
  op->tags_A.tagged = t;
  op->tags_A.l2_budget = kRingL2Budget;
  // rows by degree, largest first: the row groups of one warp (narrow slabs)
  // then get rows of about the same length
  int32_t maxd = 0;
  for (int64_t i = 0; i < op->n; ++i) maxd = std::max(maxd, rp[i + 1] - rp[i]);
  std::vector<int64_t> pos((size_t)maxd + 1, 0);
  for (int64_t i = 0; i < op->n; ++i) pos[rp[i + 1] - rp[i]] += 1;
  int64_t acc = 0;
  for (int64_t d = maxd; d >= 0; --d) {
    const int64_t c = pos[d];
    pos[d] = acc;
    acc += c;
  }
  std::vector<int32_t> order((size_t)op->n);
  for (int64_t i = 0; i < op->n; ++i) order[pos[rp[i + 1] - rp[i]]++] = (int32_t)i;
  int32_t *o = (int32_t *)owned_alloc(op, sizeof(int32_t) * op->n, s);
  if (!o) return fail(ISVD_ERR_WORKSPACE, "row order allocation failed");
  ISVD_CUDA_TRY(cudaMemcpyAsync(o, order.data(), sizeof(int32_t) * op->n, cudaMemcpyHostToDevice, s));
  ISVD_CUDA_TRY(cudaStreamSynchronize(s));
  op->tags_A.row_order = o;
  return ISVD_OK;
}

// Nonzero-chunk plan: row of every nonzero (device), rows that cross a chunk
// boundary and rows without nonzeros (host lists, uploaded).
isvd_status build_chunks(isvd_operator *op, const int32_t *rowptr_dev, int64_t rows, int64_t nnz, ChunkPlan *cp,
                         cudaStream_t s) {
  free_chunks(op, cp, s);
  cp->nnz = nnz;
  cp->CH = op->chunk_nnz;
  cp->nchunks = nnz > 0 ? ceil_div(nnz, cp->CH) : 0;
  if (nnz > 0) {
    cp->row_of = (int32_t *)op_alloc(op, sizeof(int32_t) * nnz, s);
    if (!cp->row_of) return fail(ISVD_ERR_WORKSPACE, "row index allocation failed");
    row_of_entry_kernel<<<grid_for(rows), 256, 0, s>>>(rows, rowptr_dev, cp->row_of);
    ISVD_CUDA_TRY(cudaGetLastError());
  }
  std::vector<int32_t> rp((size_t)rows + 1);
  ISVD_CUDA_TRY(cudaMemcpyAsync(rp.data(), rowptr_dev, sizeof(int32_t) * (rows + 1), cudaMemcpyDeviceToHost, s));
  ISVD_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int4> split;
  std::vector<int32_t> empty;
  for (int64_t i = 0; i < rows; ++i) {
    const int64_t e0 = rp[i], e1 = rp[i + 1];
    if (e0 == e1) {
      empty.push_back((int32_t)i);
      continue;
    }
    const int64_t cf = e0 / cp->CH, cl = (e1 - 1) / cp->CH;
    if (cf != cl) split.push_back(make_int4((int)i, (int)cf, (int)cl, 0));
  }
  cp->nsplit = (int32_t)split.size();
  cp->nempty = (int32_t)empty.size();
  if (cp->nsplit) {
    cp->split = (int4 *)op_alloc(op, sizeof(int4) * split.size(), s);
    if (!cp->split) return fail(ISVD_ERR_WORKSPACE, "split-row list allocation failed");
    ISVD_CUDA_TRY(cudaMemcpyAsync(cp->split, split.data(), sizeof(int4) * split.size(), cudaMemcpyHostToDevice, s));
  }
  if (cp->nempty) {
    cp->empty = (int32_t *)op_alloc(op, sizeof(int32_t) * empty.size(), s);
    if (!cp->empty) return fail(ISVD_ERR_WORKSPACE, "empty-row list allocation failed");
    ISVD_CUDA_TRY(cudaMemcpyAsync(cp->empty, empty.data(), sizeof(int32_t) * empty.size(), cudaMemcpyHostToDevice, s));
  }
  ISVD_CUDA_TRY(cudaStreamSynchronize(s));
  return ISVD_OK;
}

isvd_status check_csr_host(const isvd_csr &m, const char *name) {
  if (m.rows < 1 || m.cols < 1) return fail(ISVD_ERR_INVALID_ARGUMENT, "%s: empty shape", name);
  if (m.nnz < 0 || m.nnz >= ((int64_t)1 << 31)) return fail(ISVD_ERR_INVALID_ARGUMENT, "%s: nnz out of range", name);
  if (m.rows >= ((int64_t)1 << 31) || m.cols >= ((int64_t)1 << 31))
    return fail(ISVD_ERR_INVALID_ARGUMENT, "%s: dimension >= 2^31", name);
  if (!m.rowptr || (m.nnz > 0 && !m.colidx)) return fail(ISVD_ERR_INVALID_ARGUMENT, "%s: null CSR array", name);
  return ISVD_OK;
}

isvd_status validate_csr_dev(isvd_operator *op, const isvd_csr &m, int32_t *flags, const char *name, cudaStream_t s) {
  ISVD_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int32_t) * 8, s));
  validate_csr_kernel<<<grid_for(std::max(m.rows + 1, m.nnz)), 256, 0, s>>>(m.rows, m.cols, m.nnz, m.rowptr,
                                                                            m.colidx, m.values, flags);
  ISVD_CUDA_TRY(cudaGetLastError());
  int32_t h[8];
  ISVD_CUDA_TRY(cudaMemcpyAsync(h, flags, sizeof h, cudaMemcpyDeviceToHost, s));
  ISVD_CUDA_TRY(cudaStreamSynchronize(s));
  (void)op;
  if (h[0]) return fail(ISVD_ERR_INVALID_GRAPH, "%s: rowptr is not a valid CSR row pointer", name);
  if (h[1]) return fail(ISVD_ERR_INVALID_GRAPH, "%s: column index out of range", name);
  if (h[2]) return fail(ISVD_ERR_INVALID_GRAPH, "%s: non-finite value", name);
  return ISVD_OK;
}

// Stable transpose of a CSR (rows x cols) into (cols x rows) with explicit values.
isvd_status transpose_csr(isvd_operator *op, int64_t rows, int64_t cols, int64_t nnz, const int32_t *rowptr,
                          const int32_t *colidx, const float *values, int32_t **t_rowptr, int32_t **t_colidx,
                          float **t_values, cudaStream_t s) {
  Scratch sc{op, s, {}};
  int32_t *keys_out = (int32_t *)sc.get(sizeof(int32_t) * nnz);
  int32_t *idx_in = (int32_t *)sc.get(sizeof(int32_t) * nnz);
  int32_t *idx_out = (int32_t *)sc.get(sizeof(int32_t) * nnz);
  int32_t *row_of = (int32_t *)sc.get(sizeof(int32_t) * nnz);
  int32_t *counts = (int32_t *)sc.get(sizeof(int32_t) * (cols + 1));
  *t_rowptr = (int32_t *)owned_alloc(op, sizeof(int32_t) * (cols + 1), s);
  *t_colidx = (int32_t *)owned_alloc(op, sizeof(int32_t) * nnz, s);
  *t_values = (float *)owned_alloc(op, sizeof(float) * nnz, s);
  if (!keys_out || !idx_in || !idx_out || !row_of || !counts || !*t_rowptr || !*t_colidx || !*t_values)
    return fail(ISVD_ERR_WORKSPACE, "transpose workspace allocation failed");
  iota_kernel<<<grid_for(nnz), 256, 0, s>>>(nnz, idx_in);
  row_of_entry_kernel<<<grid_for(rows), 256, 0, s>>>(rows, rowptr, row_of);
  ISVD_CUDA_TRY(cudaGetLastError());
  size_t tmp_bytes = 0;
  const int end_bit = bits_for((uint64_t)cols);
  ISVD_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, colidx, keys_out, idx_in, idx_out, (int)nnz, 0,
                                                end_bit, s));
  void *tmp = sc.get(tmp_bytes);
  if (!tmp) return fail(ISVD_ERR_WORKSPACE, "sort workspace allocation failed");
  ISVD_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, colidx, keys_out, idx_in, idx_out, (int)nnz, 0,
                                                end_bit, s));
  gather_transpose_kernel<<<grid_for(nnz), 256, 0, s>>>(nnz, idx_out, row_of, values, *t_colidx, *t_values);
  ISVD_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int32_t) * (cols + 1), s));
  count_kernel<<<grid_for(nnz), 256, 0, s>>>(nnz, keys_out, counts);
  ISVD_CUDA_TRY(cudaGetLastError());
  size_t scan_bytes = 0;
  ISVD_CUDA_TRY(cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, counts, *t_rowptr, (int)(cols + 1), s));
  void *tmp2 = sc.get(scan_bytes);
  if (!tmp2) return fail(ISVD_ERR_WORKSPACE, "scan workspace allocation failed");
  ISVD_CUDA_TRY(cub::DeviceScan::ExclusiveSum(tmp2, scan_bytes, counts, *t_rowptr, (int)(cols + 1), s));
  ISVD_CUDA_TRY(cudaStreamSynchronize(s));
  return ISVD_OK;
}

// A == A^T (pattern and values) by sorting the (row, col) and (col, row) keys.
isvd_status check_symmetry(isvd_operator *op, const isvd_csr &A, int32_t *flags, cudaStream_t s) {
  const int64_t nnz = A.nnz, n = A.rows;
  if (nnz == 0) return ISVD_OK;
  Scratch sc{op, s, {}};
  uint64_t *ka = (uint64_t *)sc.get(sizeof(uint64_t) * nnz);
  uint64_t *kb = (uint64_t *)sc.get(sizeof(uint64_t) * nnz);
  uint64_t *ka2 = (uint64_t *)sc.get(sizeof(uint64_t) * nnz);
  uint64_t *kb2 = (uint64_t *)sc.get(sizeof(uint64_t) * nnz);
  float *va = nullptr, *vb = nullptr;
  if (A.values) {
    va = (float *)sc.get(sizeof(float) * nnz);
    vb = (float *)sc.get(sizeof(float) * nnz);
  }
  if (!ka || !kb || !ka2 || !kb2 || (A.values && (!va || !vb)))
    return fail(ISVD_ERR_WORKSPACE, "symmetry-check workspace allocation failed");
  edge_keys_kernel<<<grid_for(n), 256, 0, s>>>(n, nnz, A.rowptr, A.colidx, ka, kb);
  ISVD_CUDA_TRY(cudaGetLastError());
  const int end_bit = bits_for((uint64_t)n * (uint64_t)n);
  size_t tmp_bytes = 0;
  if (A.values)
    ISVD_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, ka, ka2, A.values, va, (int)nnz, 0, end_bit, s));
  else
    ISVD_CUDA_TRY(cub::DeviceRadixSort::SortKeys(nullptr, tmp_bytes, ka, ka2, (int)nnz, 0, end_bit, s));
  void *tmp = sc.get(tmp_bytes);
  if (!tmp) return fail(ISVD_ERR_WORKSPACE, "sort workspace allocation failed");
  if (A.values) {
    ISVD_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, ka, ka2, A.values, va, (int)nnz, 0, end_bit, s));
    ISVD_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, kb, kb2, A.values, vb, (int)nnz, 0, end_bit, s));
  } else {
    ISVD_CUDA_TRY(cub::DeviceRadixSort::SortKeys(tmp, tmp_bytes, ka, ka2, (int)nnz, 0, end_bit, s));
    ISVD_CUDA_TRY(cub::DeviceRadixSort::SortKeys(tmp, tmp_bytes, kb, kb2, (int)nnz, 0, end_bit, s));
  }
  ISVD_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int32_t) * 8, s));
  compare_kernel<<<grid_for(nnz), 256, 0, s>>>(nnz, ka2, kb2, va, vb, flags);
  ISVD_CUDA_TRY(cudaGetLastError());
  int32_t h[8];
  ISVD_CUDA_TRY(cudaMemcpyAsync(h, flags, sizeof h, cudaMemcpyDeviceToHost, s));
  ISVD_CUDA_TRY(cudaStreamSynchronize(s));
  if (h[4]) return fail(ISVD_ERR_INVALID_GRAPH, "A is not symmetric (pattern or values)");
  return ISVD_OK;
}

isvd_status create_impl(const isvd_operator_desc *desc, isvd_operator *op, cudaStream_t s) {
  const isvd_operator_desc &d = *desc;
  ISVD_TRY(check_csr_host(d.A, "A"));
  if (d.A.rows != d.A.cols) return fail(ISVD_ERR_SHAPE, "A must be square");
  if (d.norm != ISVD_NORM_ROW && d.norm != ISVD_NORM_SYM_SELFLOOP && d.norm != ISVD_NORM_SYM_NOSELF)
    return fail(ISVD_ERR_INVALID_ARGUMENT, "unknown normalisation %d", (int)d.norm);
  op->n = d.A.rows;
  if (d.form == ISVD_FORM_POLY) {
    if (d.degree < 1 || d.degree > ISVD_MAX_DEGREE)
      return fail(ISVD_ERR_INVALID_ARGUMENT, "degree must be in 1..%d", ISVD_MAX_DEGREE);
    if (!d.coeffs) return fail(ISVD_ERR_INVALID_ARGUMENT, "coeffs is null");
    if (d.lr_rank < 0 || d.lr_rank > ISVD_MAX_LOWRANK - 1)
      return fail(ISVD_ERR_INVALID_ARGUMENT, "lr_rank must be in 0..%d", ISVD_MAX_LOWRANK - 1);
    if (d.lr_rank > 0 && (!d.lr_u || !d.lr_v || !d.lr_alpha))
      return fail(ISVD_ERR_INVALID_ARGUMENT, "low-rank factors are null");
    if (!std::isfinite(d.ones_coeff) || !std::isfinite(d.adj_coeff))
      return fail(ISVD_ERR_INVALID_ARGUMENT, "non-finite coefficient");
    op->coeffs.assign(d.coeffs, d.coeffs + d.degree);
    for (double c : op->coeffs)
      if (!std::isfinite(c)) return fail(ISVD_ERR_INVALID_ARGUMENT, "non-finite polynomial coefficient");
    if (d.lr_rank > 0) op->lr_alpha.assign(d.lr_alpha, d.lr_alpha + d.lr_rank);
    op->rows = op->cols = op->n;
  } else if (d.form == ISVD_FORM_CONCAT) {
    if (d.L < 0 || d.L > 8) return fail(ISVD_ERR_INVALID_ARGUMENT, "L must be in 0..8");
    if (d.d < 1) return fail(ISVD_ERR_INVALID_ARGUMENT, "feature width d must be >= 1");
    if (d.ones_coeff != 0.0 || d.adj_coeff != 0.0 || d.lr_rank != 0)
      return fail(ISVD_ERR_UNSUPPORTED, "corrections are only implemented for the polynomial form");
    const bool sparse = d.X.rowptr != nullptr;
    if (sparse == (d.X_dense != nullptr)) return fail(ISVD_ERR_INVALID_ARGUMENT, "give exactly one of X (CSR) and X_dense");
    if (sparse) {
      ISVD_TRY(check_csr_host(d.X, "X"));
      if (d.X.rows != op->n || d.X.cols != d.d) return fail(ISVD_ERR_SHAPE, "X must be n x d");
    } else if (op->n * d.d >= ((int64_t)1 << 31)) {
      return fail(ISVD_ERR_UNSUPPORTED, "dense X with n*d >= 2^31 entries");
    }
    op->rows = op->n;
    op->cols = d.d * (d.L + 1);
  } else {
    return fail(ISVD_ERR_INVALID_ARGUMENT, "unknown form %d", (int)d.form);
  }
  if (d.gather_rows) {
    if (d.n_gather < 1 || d.n_gather > op->rows)
      return fail(ISVD_ERR_INVALID_ARGUMENT, "n_gather must be in 1..%lld", (long long)op->rows);
  } else if (d.n_gather != 0) {
    return fail(ISVD_ERR_INVALID_ARGUMENT, "n_gather without gather_rows");
  }
  ISVD_CUDA_TRY(small_kernels_init());
  ISVD_CUDA_TRY(dense_kernels_init());
  ISVD_CUDA_TRY(cudaStreamCreateWithFlags(&op->capture_stream, cudaStreamNonBlocking));
  ISVD_CUDA_TRY(cudaStreamCreateWithFlags(&op->side.stream, cudaStreamNonBlocking));
  ISVD_CUDA_TRY(cudaEventCreateWithFlags(&op->side.fork, cudaEventDisableTiming));
  ISVD_CUDA_TRY(cudaEventCreateWithFlags(&op->side.join, cudaEventDisableTiming));

  const int64_t n = op->n;
  float *vecs = (float *)owned_alloc(op, sizeof(float) * 4 * n, s);
  int32_t *flags = (int32_t *)owned_alloc(op, sizeof(int32_t) * 8, s);
  if (!vecs || !flags) return fail(ISVD_ERR_WORKSPACE, "operator allocation failed");
  op->deg = vecs;
  op->inv_d = vecs + n;
  op->s = vecs + 2 * n;
  op->s2 = vecs + 3 * n;
  ISVD_TRY(validate_csr_dev(op, d.A, flags, "A", s));
  ISVD_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int32_t) * 8, s));
  degree_kernel<<<grid_for(n), 256, 0, s>>>(n, d.A.rowptr, d.A.values, d.norm == ISVD_NORM_ROW ? 1 : 0, op->deg,
                                            op->inv_d, op->s, op->s2, flags);
  ISVD_CUDA_TRY(cudaGetLastError());
  {
    int32_t h[8];
    ISVD_CUDA_TRY(cudaMemcpyAsync(h, flags, sizeof h, cudaMemcpyDeviceToHost, s));
    ISVD_CUDA_TRY(cudaStreamSynchronize(s));
    if (h[3])
      return fail(ISVD_ERR_INVALID_GRAPH,
                  "a row of A has zero (or negative) degree: T = D^-1 A is undefined (add a self-loop)");
  }
  if (!(d.flags & ISVD_FLAG_SKIP_SYMMETRY_CHECK)) ISVD_TRY(check_symmetry(op, d.A, flags, s));
  if (d.gather_rows) {
    // strictly increasing row indices inside M; the operator has n_gather rows
    ISVD_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int32_t) * 8, s));
    validate_rows_kernel<<<grid_for(d.n_gather), 256, 0, s>>>(d.gather_rows, d.n_gather, op->rows, flags);
    ISVD_CUDA_TRY(cudaGetLastError());
    int32_t h[8];
    ISVD_CUDA_TRY(cudaMemcpyAsync(h, flags, sizeof h, cudaMemcpyDeviceToHost, s));
    ISVD_CUDA_TRY(cudaStreamSynchronize(s));
    if (h[0]) return fail(ISVD_ERR_INVALID_ARGUMENT, "gather_rows must be strictly increasing indices in [0, %lld)",
                          (long long)op->rows);
    op->rows = d.n_gather;
  }
  ISVD_TRY(build_heavy(op, d.A.rowptr, n, &op->heavy_A, s));
  ISVD_TRY(build_chunks(op, d.A.rowptr, n, d.A.nnz, &op->chunk_A, s));
  ISVD_TRY(build_slab_plan(op, d.A.rowptr, n, op->heavy_A.threshold, op->heavy_A.chunk, &op->slab_A, s));
  ISVD_TRY(build_tags(op, s));

  if (d.form == ISVD_FORM_CONCAT) {
    if (d.X.rowptr) {
      ISVD_TRY(validate_csr_dev(op, d.X, flags, "X", s));
      op->x_rowptr = d.X.rowptr;
      op->x_colidx = d.X.colidx;
      op->x_values = d.X.values;
      op->x_nnz = d.X.nnz;
    } else {
      const int64_t nnz = n * d.d;
      op->xd_rowptr = (int32_t *)owned_alloc(op, sizeof(int32_t) * (n + 1), s);
      op->xd_colidx = (int32_t *)owned_alloc(op, sizeof(int32_t) * nnz, s);
      if (!op->xd_rowptr || !op->xd_colidx) return fail(ISVD_ERR_WORKSPACE, "dense-X index allocation failed");
      dense_csr_kernel<<<grid_for(nnz), 256, 0, s>>>(n, d.d, op->xd_rowptr, op->xd_colidx);
      ISVD_CUDA_TRY(cudaGetLastError());
      op->x_rowptr = op->xd_rowptr;
      op->x_colidx = op->xd_colidx;
      op->x_values = d.X_dense;
      op->x_nnz = nnz;
    }
    ISVD_TRY(transpose_csr(op, n, d.d, op->x_nnz, op->x_rowptr, op->x_colidx, op->x_values, &op->xt_rowptr,
                           &op->xt_colidx, &op->xt_values, s));
    ISVD_TRY(build_heavy(op, op->x_rowptr, n, &op->heavy_X, s));
    ISVD_TRY(build_heavy(op, op->xt_rowptr, d.d, &op->heavy_XT, s));
    ISVD_TRY(build_chunks(op, op->x_rowptr, n, op->x_nnz, &op->chunk_X, s));
    ISVD_TRY(build_chunks(op, op->xt_rowptr, d.d, op->x_nnz, &op->chunk_XT, s));
  }
  ISVD_CUDA_TRY(cudaStreamSynchronize(s));
  return ISVD_OK;
}

// ---- apply ---------------------------------------------------------------------

struct Chain {
  const isvd_operator *op;
  int dtype;
  cudaStream_t s;
  const ApplyScratch *sc;
};

int slab_cols(const isvd_operator *op, int dtype) {
  if (op->spmm_algo == 1) return chunk_slab_cols(dtype);
  if (op->spmm_algo == 2) return ring_max_cols(dtype);
  const int c = dtype == DT_F32 ? op->slab_cols_f32 : op->slab_cols_bf16;
  // the packed-slab kernel gives each lane one 16-byte chunk: at most 32 lanes' worth
  const int cap = dtype == DT_F32 ? 128 : 256;
  return op->spmm_algo == 3 && c > cap ? cap : c;
}

SpmmArgs base_args_A(const isvd_operator *op) {
  SpmmArgs a{};
  a.rows = op->n;
  a.rowptr = op->desc.A.rowptr;
  a.colidx = op->desc.A.colidx;
  a.values = op->desc.A.values;
  a.scalar = 1.f;
  a.ax_scalar = 1.f;
  a.heavy_threshold = op->heavy_A.n_chunks > 0 ? op->heavy_A.threshold : INT_MAX;
  a.cache_hints = op->cache_hints;
  a.rows_occupancy = op->rows_occupancy;
  a.prefetch = op->prefetch;
  return a;
}

int slabs_needed(int dtype, int32_t b, int32_t scols);

// fill slabs for one segment of width b; false when they do not fit kMaxSlabs
//
// pack_in / pack_out: `in` / `out` hold the block slab by slab, each slab a
// dense [rows][w] block (w = its width rounded up to 16 bytes) following the
// previous one; ldi / ldo are then ignored.
bool add_slabs(SpmmArgs &a, int dtype, int32_t b, int32_t scols, int32_t col_base, const void *in, int64_t ldi,
               void *out, int64_t ldo, const void *axpy, int64_t lda, bool pack_in = false,
               bool pack_out = false) {
  SpmmSlab tmp[256];
  int ns = 0;
  if (scols == ring_max_cols(dtype)) {  // ring form: full-width slabs
    for (int32_t c0 = 0; c0 < b && ns < 256; c0 += scols) {
      SpmmSlab sl{};
      sl.col0 = c0;
      sl.width = (b - c0) < scols ? (b - c0) : scols;
      sl.group = 32;
      tmp[ns++] = sl;
    }
  } else {
    if (slabs_needed(dtype, b, scols) > 256) return false;
    ns = make_slabs(dtype, b, scols, tmp);
  }
  if (a.nslabs + ns > kMaxSlabs) return false;
  const size_t es = dtype_size(dtype);
  const int64_t vn = 16 / (int64_t)es;
  size_t packed_off = 0;  // elements before this slab in a packed block
  for (int i = 0; i < ns; ++i) {
    SpmmSlab sl = tmp[i];
    const int64_t pw = round_up(sl.width, vn);
    sl.in = pack_in ? (const char *)in + packed_off * es : (const char *)in + (size_t)sl.col0 * es;
    sl.ldi = pack_in ? pw : ldi;
    sl.out = pack_out ? (char *)out + packed_off * es : (char *)out + (size_t)sl.col0 * es;
    sl.ldo = pack_out ? pw : ldo;
    packed_off += (size_t)a.rows * (size_t)pw;
    sl.axpy = axpy ? (const char *)axpy + (size_t)sl.col0 * es : nullptr;
    sl.lda = lda;
    sl.col0 += col_base;
    a.slab[a.nslabs++] = sl;
  }
  return true;
}

#define ISVD_SLABS(call) \
  do {                                                                                      \
    if (!(call)) return fail(ISVD_ERR_UNSUPPORTED, "block too wide for the sparse-product kernel"); \
  } while (0)

int slabs_needed(int dtype, int32_t b, int32_t scols) {
  const int vn = dtype == DT_F32 ? 4 : 8;
  const int cap = scols == ring_max_cols(dtype) ? scols : 64 * vn;  // ring slabs span the full width
  int sc = scols > cap ? cap : scols;
  return (int)ceil_div(b, sc);
}

cudaError_t run(const Chain &c, SpmmArgs &a, const HeavyPlan &hp, const ChunkPlan &cp, int64_t pw) {
  if (a.colidx == c.op->desc.A.colidx) a.row_order = c.op->tags_A.row_order;
  if (c.op->spmm_algo == 2) {
    static const RingTags none;
    const RingTags &tags = a.colidx == c.op->desc.A.colidx ? c.op->tags_A : none;
    for (int i = 0; i < a.nslabs; ++i) {
      SpmmArgs one = a;
      one.slab[0] = a.slab[i];
      one.nslabs = 1;
      const cudaError_t e = spmm_ring_launch(one, c.dtype, cp, tags, c.sc->heavy_partial, pw, c.s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (c.op->spmm_algo == 1) return spmm_chunk_launch(a, c.dtype, cp, c.sc->heavy_partial, pw, c.s);
  if (c.op->spmm_algo == 3 && a.colidx == c.op->desc.A.colidx)
    return spmm_slab_launch(a, c.dtype, c.op->slab_A, c.sc->heavy_partial, pw, c.s);
  if (a.cache_hints && c.op->hot_tags && a.colidx == c.op->desc.A.colidx && c.op->tags_A.tagged) {
    // per slab: the hottest degree buckets whose gathered rows fit the L2 budget keep priority
    const RingTags &t = c.op->tags_A;
    a.tagged = t.tagged;
    for (int i = 0; i < a.nslabs; ++i) {
      const double row_bytes = (double)round_up((int64_t)a.slab[i].width * (int64_t)dtype_size(c.dtype), 32);
      double bytes = 0.0;
      int hb = 32;
      while (hb > 0 && bytes + (double)t.hist[hb - 1] * row_bytes <= (double)t.l2_budget) {
        bytes += (double)t.hist[hb - 1] * row_bytes;
        --hb;
      }
      a.slab[i].hot_bucket = hb;
    }
  }
  return spmm_launch(a, c.dtype, hp, c.sc->heavy_partial, pw, c.s, c.op->side);
}

int64_t partial_rows(const isvd_operator *op) {
  return std::max<int64_t>({op->heavy_A.n_chunks, op->heavy_X.n_chunks, op->heavy_XT.n_chunks, op->slab_A.n_slots,
                            2 * op->chunk_A.nchunks, 2 * op->chunk_X.nchunks, 2 * op->chunk_XT.nchunks, 1});
}

}  // namespace

// Rows of a composite's two block temporaries: the node's own rows and
// columns and those of each child (the intermediates of a product).
static int64_t composite_span(const isvd_operator *op) {
  int64_t m = std::max(op->rows, op->cols);
  for (const isvd_operator *c : op->child) m = std::max(m, std::max(c->rows, c->cols));
  return m;
}

// Largest row count of any product in the tree (a cache slot's rows).
static int64_t tree_span(const isvd_operator *op) {
  int64_t m = std::max(op->rows, op->cols);
  for (const isvd_operator *c : op->child) m = std::max(m, tree_span(c));
  return m;
}

static size_t cache_slot_bytes(const isvd_operator *op, int32_t b, int dtype) {
  return (size_t)round_up((int64_t)(dtype_size(dtype) * tree_span(op) * round_up(b, 8)), 256);
}

// Scratch of a composite evaluated as a child (no cache region of its own).
static size_t composite_core_bytes(const isvd_operator *op, int32_t b, int dtype, bool transpose) {
  const size_t es = dtype_size(dtype);
  const int64_t bseg = round_up(b, 8);
  // two temporaries, then one region the children use in turn
  const size_t t = (size_t)round_up((int64_t)(es * composite_span(op) * bseg), 256);
  size_t cmax = 0;
  for (const isvd_operator *c : op->child)
    cmax = std::max(cmax, c->compose >= 0 ? composite_core_bytes(c, b, dtype, transpose)
                                          : apply_scratch_bytes(c, b, dtype, transpose));
  return 2 * t + cmax;
}

size_t apply_scratch_bytes(const isvd_operator *op, int32_t b, int dtype, bool transpose) {
  const size_t es = dtype_size(dtype);
  const int64_t bseg = round_up(b, 8);
  if (op->compose >= 0) {
    // as the root of an evaluation: the slots of its lazy product cache follow
    const size_t slots = op->cache_on ? op->cache_keys[transpose ? 1 : 0].size() : 0;
    return composite_core_bytes(op, b, dtype, transpose) + slots * cache_slot_bytes(op, b, dtype);
  }
  size_t total = 0;
  auto add = [&](size_t x) { total += (size_t)round_up((int64_t)x, 256); };
  add(es * op->n * bseg);  // z1
  add(es * op->n * bseg);  // z2
  int64_t pw = bseg;
  if (op->desc.form == ISVD_FORM_CONCAT) {
    add(es * op->n * bseg * (op->desc.L + 1));  // P
    pw = bseg * (op->desc.L + 1);
  }
  const int r = (op->desc.ones_coeff != 0.0 ? 1 : 0) + op->desc.lr_rank;
  add(sizeof(float) * (size_t)std::max(r, 1) * bseg);
  add(sizeof(double) * (size_t)lowrank_partials(op->n) * std::max(r, 1) * bseg);
  const int64_t chunks = partial_rows(op);
  add(sizeof(float) * (size_t)chunks * pw);
  if (op->desc.form == ISVD_FORM_CONCAT && op->desc.X_dense)
    add(xdense_scratch_bytes((int32_t)op->desc.d, op->desc.L + 1, (int32_t)bseg, op->n));
  if (op->desc.gather_rows) add(es * op->n * bseg);  // gz
  return total;
}

void apply_scratch_carve(const isvd_operator *op, int32_t b, int dtype, bool transpose, char *base,
                         ApplyScratch *sc) {
  (void)transpose;
  const size_t es = dtype_size(dtype);
  const int64_t bseg = round_up(b, 8);
  if (op->compose >= 0) {
    const size_t t = (size_t)round_up((int64_t)(es * composite_span(op) * bseg), 256);
    sc->ct1 = base;
    sc->ct2 = base + t;
    sc->child_base = base + 2 * t;
    sc->cache_base = base + composite_core_bytes(op, b, dtype, transpose);
    sc->cache_slot_bytes = cache_slot_bytes(op, b, dtype);
    return;
  }
  size_t off = 0;
  auto take = [&](size_t x) {
    char *p = base + off;
    off += (size_t)round_up((int64_t)x, 256);
    return p;
  };
  sc->z1 = take(es * op->n * bseg);
  sc->z2 = take(es * op->n * bseg);
  if (op->desc.form == ISVD_FORM_CONCAT) sc->p = take(es * op->n * bseg * (op->desc.L + 1));
  const int r = (op->desc.ones_coeff != 0.0 ? 1 : 0) + op->desc.lr_rank;
  sc->lr_c = (float *)take(sizeof(float) * (size_t)std::max(r, 1) * bseg);
  sc->lr_partial = (double *)take(sizeof(double) * (size_t)lowrank_partials(op->n) * std::max(r, 1) * bseg);
  int64_t pw = op->desc.form == ISVD_FORM_CONCAT ? bseg * (op->desc.L + 1) : bseg;
  const int64_t chunks = partial_rows(op);
  sc->heavy_partial = (float *)take(sizeof(float) * (size_t)chunks * pw);
  if (op->desc.form == ISVD_FORM_CONCAT && op->desc.X_dense)
    sc->xdense = take(xdense_scratch_bytes((int32_t)op->desc.d, op->desc.L + 1, (int32_t)bseg, op->n));
  if (op->desc.gather_rows) sc->gz = take(es * op->n * bseg);
}

// Horner evaluation of sum_{k=1..K} c_k N^k G (+ corrections), Eq. 3 with the
// products taken right to left (Sec. 4; App. A.3's lazy cache is subsumed:
// K sparse products per apply).  N^T for N = D^-1 A is A D^-1 (A symmetric),
// evaluated on D^-1-scaled iterates; Â is symmetric and evaluated on
// (D+I)^-1/2-scaled iterates so that only the first product gathers a weight.
// Â - (D+I)^-1 (label re-use, Sec. 5.3) is Â without its identity term.
static isvd_status apply_poly(isvd_operator *op, const void *G, int64_t ldg, int32_t b, void *out, int64_t ldo,
                              int dtype, bool transpose, const ApplyScratch &sc, cudaStream_t s) {
  const isvd_operator_desc &d = op->desc;
  const int K = d.degree;
  const std::vector<double> &c = op->coeffs;  // c[k-1] = c_k
  const bool row = d.norm == ISVD_NORM_ROW;
  const int32_t selfloop = d.norm == ISVD_NORM_SYM_SELFLOOP ? 1 : 0;  // Â's identity term
  const int64_t bseg = round_up(b, 8);
  const int scols = slab_cols(op, dtype);
  const Chain ch{op, dtype, s, &sc};

  // corrections: c = V^T G with the all-ones vector first (transpose swaps u and v)
  const int ones = d.ones_coeff != 0.0 ? 1 : 0;
  const int r = ones + d.lr_rank;
  if (r > 0 && ones && d.lr_rank == 0 && sc.ones_parts) {
    // 1^T G from the column sums that the step writing G formed
    ISVD_CUDA_TRY(colsum_reduce_launch(sc.ones_parts, sc.ones_nparts, sc.ones_ld, b, (int32_t)bseg, sc.lr_c, s));
  } else if (r > 0) {
    const float *V = transpose ? d.lr_u : d.lr_v;
    ISVD_CUDA_TRY(lowrank_project_launch(G, ldg, dtype, op->n, b, d.lr_rank ? V : nullptr, d.lr_rank, r, ones,
                                         sc.lr_partial, lowrank_partials(op->n), sc.lr_c, bseg, s));
  }
  auto set_lowrank = [&](SpmmArgs &a) {
    if (r == 0) return;
    a.lr_rank = r;
    a.lr_ones_first = ones;
    a.lr_u = d.lr_rank ? (transpose ? d.lr_v : d.lr_u) : nullptr;
    a.lr_ldu = d.lr_rank;
    a.lr_c = sc.lr_c;
    a.lr_ldc = bseg;
    int t = 0;
    if (ones) a.lr_alpha[t++] = (float)d.ones_coeff;
    for (int q = 0; q < d.lr_rank; ++q) a.lr_alpha[t++] = (float)op->lr_alpha[q];
  };

  const void *cur = G;
  int64_t ldcur = ldg;
  void *bufs[2] = {sc.z1, sc.z2};
  int which = 0;
  for (int step = K; step >= 1; --step) {
    // step k computes Z_{k-1}-like iterate: first step (k == K) consumes G itself
    const bool first = step == K;
    const bool last = step == 1;
    SpmmArgs a = base_args_A(op);
    a.scalar = first ? (float)c[K - 1] : 1.f;
    void *dst = last ? out : bufs[which];
    const int64_t lddst = last ? ldo : bseg;
    const void *axp = nullptr;
    if (!last) {
      axp = G;
      a.ax_scalar = (float)c[step - 2];
    }
    if (row && !transpose) {
      a.rowscale = op->inv_d;
    } else if (row && transpose) {
      if (first) a.colw = op->inv_d;
      a.rowscale = last ? nullptr : op->inv_d;
      a.ax_rowscale = op->inv_d;
    } else {  // Â
      if (first) a.colw = op->s;
      a.self_term = selfloop;
      a.rowscale = last ? op->s : op->s2;
      a.ax_rowscale = op->s;
    }
    if (last) set_lowrank(a);
    // packed temporaries: every iterate between two products is written and
    // gathered slab by slab (the row kernel only)
    const bool pack = (op->packed_temps && op->spmm_algo == 0) || op->spmm_algo == 3;
    ISVD_SLABS(add_slabs(a, dtype, b, scols, 0, cur, ldcur, dst, lddst, axp, ldg, pack && !first, pack && !last));
    ISVD_CUDA_TRY(run(ch, a, op->heavy_A, op->chunk_A, bseg));
    cur = dst;
    ldcur = lddst;
    which ^= 1;
  }
  if (d.adj_coeff != 0.0) {
    // + beta A G  (A symmetric, so the same for the transpose)
    SpmmArgs a = base_args_A(op);
    a.scalar = (float)d.adj_coeff;
    a.ax_scalar = 1.f;
    ISVD_SLABS(add_slabs(a, dtype, b, scols, 0, G, ldg, out, ldo, out, ldo));
    ISVD_CUDA_TRY(run(ch, a, op->heavy_A, op->chunk_A, bseg));
  }
  return ISVD_OK;
}

// M = [X | N X | ... | N^L X] (Eq. 6).  M G = sum_l N^l X G_l evaluated as
// P = X [G_0 | ... | G_L] (one sparse product over all blocks), then Horner
// Y = P_L, Y <- P_l + N Y.  M^T H = [X^T H ; X^T N^T H ; ...]: the iterates
// N^T^l H are stacked side by side and X^T is applied once to all of them.
static isvd_status apply_concat(isvd_operator *op, const void *G, int64_t ldg, int32_t b, void *out, int64_t ldo,
                                int dtype, bool transpose, const ApplyScratch &sc, cudaStream_t s) {
  const isvd_operator_desc &d = op->desc;
  const int L = d.L;
  const bool row = d.norm == ISVD_NORM_ROW;
  const int32_t selfloop = d.norm == ISVD_NORM_SYM_SELFLOOP ? 1 : 0;  // Â's identity term
  const int64_t bseg = round_up(b, 8);
  const int64_t ldp = bseg * (L + 1);
  const size_t es = dtype_size(dtype);
  const int scols = slab_cols(op, dtype);
  const Chain ch{op, dtype, s, &sc};
  if ((int64_t)(L + 1) * slabs_needed(dtype, b, scols) > kMaxSlabs)
    return fail(ISVD_ERR_UNSUPPORTED, "block too wide for the stacked feature product (L+1 = %d, b = %d)", L + 1, b);
  char *P = (char *)sc.p;
  auto seg = [&](int l) { return P + (size_t)l * bseg * es; };

  // dense X: small dense products instead of the X-as-CSR sparse ones
  const bool xd = d.X_dense && d.d <= ISVD_MAX_BLOCK && (int64_t)(L + 1) * bseg <= ISVD_MAX_BLOCK && sc.xdense;
  if (!transpose && xd) {
    // P = X [G_0 | ... | G_L] (or out = X G_0 when L = 0: only the b columns of out)
    ISVD_CUDA_TRY(xdense_forward(d.X_dense, op->n, (int32_t)d.d, G, ldg, dtype, b, (int32_t)bseg, L + 1,
                                 L == 0 ? out : (void *)P, L == 0 ? ldo : ldp, sc.xdense, s));
  }
  if (!transpose) {
    // P_l = X G_l
    SpmmArgs ax{};
    ax.rows = op->n;
    ax.rowptr = op->x_rowptr;
    ax.colidx = op->x_colidx;
    ax.values = op->x_values;
    ax.scalar = 1.f;
    ax.ax_scalar = 1.f;
    ax.heavy_threshold = op->heavy_X.n_chunks > 0 ? op->heavy_X.threshold : INT_MAX;
    ax.cache_hints = op->cache_hints;
    ax.rows_occupancy = op->rows_occupancy;
    ax.prefetch = op->prefetch;
    if (!xd) {
      for (int l = 0; l <= L; ++l) {
        const char *gin = (const char *)G + (size_t)l * d.d * ldg * es;
        if (L == 0) ISVD_SLABS(add_slabs(ax, dtype, b, scols, 0, gin, ldg, out, ldo, nullptr, 0));
        else ISVD_SLABS(add_slabs(ax, dtype, b, scols, (int32_t)(l * bseg), gin, ldg, seg(l), ldp, nullptr, 0));
      }
      ISVD_CUDA_TRY(run(ch, ax, op->heavy_X, op->chunk_X, ldp));
    }
    if (L == 0) return ISVD_OK;
    // Horner over N
    const void *cur = seg(L);
    int64_t ldcur = ldp;
    void *bufs[2] = {sc.z1, sc.z2};
    int which = 0;
    for (int l = L - 1; l >= 0; --l) {
      const bool first = l == L - 1, last = l == 0;
      SpmmArgs a = base_args_A(op);
      void *dst = last ? out : bufs[which];
      const int64_t lddst = last ? ldo : bseg;
      if (row) {
        a.rowscale = op->inv_d;
      } else {
        if (first) a.colw = op->s;
        a.self_term = selfloop;
        a.rowscale = last ? op->s : op->s2;
        a.ax_rowscale = last ? nullptr : op->s;
      }
      ISVD_SLABS(add_slabs(a, dtype, b, scols, 0, cur, ldcur, dst, lddst, seg(l), ldp));
      ISVD_CUDA_TRY(run(ch, a, op->heavy_A, op->chunk_A, bseg));
      cur = dst;
      ldcur = lddst;
      which ^= 1;
    }
    return ISVD_OK;
  }
  // transpose: Q_0 = H, Q_l = N^T Q_{l-1} into P's segments
  const void *cur = G;
  int64_t ldcur = ldg;
  for (int l = 1; l <= L; ++l) {
    SpmmArgs a = base_args_A(op);
    if (row) {
      a.colw = op->inv_d;  // T^T = A D^-1
    } else {
      a.colw = op->s;
      a.self_term = selfloop;
      a.rowscale = op->s;
    }
    ISVD_SLABS(add_slabs(a, dtype, b, scols, 0, cur, ldcur, seg(l), ldp, nullptr, 0));
    ISVD_CUDA_TRY(run(ch, a, op->heavy_A, op->chunk_A, bseg));
    cur = seg(l);
    ldcur = ldp;
  }
  if (xd && dtype == DT_F32) {
    ISVD_CUDA_TRY(xdense_transpose(d.X_dense, op->n, (int32_t)d.d, (const float *)G, ldg, b, (int32_t)bseg, L + 1,
                                   (float *)P, ldp, (float *)out, ldo, sc.xdense, s));
    return ISVD_OK;
  }
  SpmmArgs at{};
  at.rows = d.d;
  at.rowptr = op->xt_rowptr;
  at.colidx = op->xt_colidx;
  at.values = op->xt_values;
  at.scalar = 1.f;
  at.ax_scalar = 1.f;
  at.heavy_threshold = op->heavy_XT.n_chunks > 0 ? op->heavy_XT.threshold : INT_MAX;
  at.cache_hints = op->cache_hints;
  at.rows_occupancy = op->rows_occupancy;
  at.prefetch = op->prefetch;
  for (int l = 0; l <= L; ++l) {
    const void *in = l == 0 ? G : (const void *)seg(l);
    const int64_t ldi = l == 0 ? ldg : ldp;
    char *o = (char *)out + (size_t)l * d.d * ldo * es;
    ISVD_SLABS(add_slabs(at, dtype, b, scols, (int32_t)(l * bseg), in, ldi, o, ldo, nullptr, 0));
  }
  ISVD_CUDA_TRY(run(ch, at, op->heavy_XT, op->chunk_XT, ldp));
  return ISVD_OK;
}

static isvd_status apply_form(isvd_operator *op, const void *G, int64_t ldg, int32_t b, void *out, int64_t ldo,
                              int dtype, bool transpose, const ApplyScratch &sc, cudaStream_t s) {
  if (op->desc.form == ISVD_FORM_POLY) return apply_poly(op, G, ldg, b, out, ldo, dtype, transpose, sc, s);
  return apply_concat(op, G, ldg, b, out, ldo, dtype, transpose, sc, s);
}

static cudaError_t gather_launch(const void *src, int64_t lds, const int32_t *idx, int64_t count, int32_t b,
                                 void *dst, int64_t ldd, bool scatter, int dtype, cudaStream_t s) {
  const unsigned grid = (unsigned)std::min<int64_t>(std::max<int64_t>(ceil_div(count * b, 256), 1), kNumSMs * 16);
  if (dtype == DT_F32)
    gather_rows_kernel<float><<<grid, 256, 0, s>>>((const float *)src, lds, idx, count, b, (float *)dst, ldd,
                                                   scatter ? 1 : 0);
  else
    gather_rows_kernel<uint16_t><<<grid, 256, 0, s>>>((const uint16_t *)src, lds, idx, count, b, (uint16_t *)dst,
                                                      ldd, scatter ? 1 : 0);
  return cudaGetLastError();
}

static cudaError_t axpy_launch(const void *x, int64_t ldx, void *y, int64_t ldy, int64_t rows, int32_t b, double w,
                               bool first, int dtype, cudaStream_t s) {
  if (rows * b == 0) return cudaSuccess;
  const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(rows * b, 256), kNumSMs * 16);
  if (dtype == DT_F32)
    axpy_block_kernel<float><<<grid, 256, 0, s>>>((const float *)x, ldx, (float *)y, ldy, rows, b, (float)w,
                                                  first ? 1 : 0);
  else
    axpy_block_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>((const __nv_bfloat16 *)x, ldx, (__nv_bfloat16 *)y, ldy,
                                                          rows, b, (float)w, first ? 1 : 0);
  return cudaGetLastError();
}

// Identity of a product during one evaluation of a composite tree (the lazy
// cache of App. A.3): the root's input is token 1; a child applied to the
// input with token t gives the product with token key(child, t, transpose);
// the rows of an input from row `off` on (the block of a concatenation's
// child) have token slice(t, off).  Equal tokens are the same matrix.
static uint64_t mix64(uint64_t x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}
static uint64_t product_key(const isvd_operator *c, uint64_t tok, bool transpose) {
  return mix64(mix64(tok ^ 0x9e3779b97f4a7c15ull) + c->serial * 2 + (transpose ? 1 : 0));
}
static uint64_t slice_token(uint64_t tok, int64_t off) {
  return mix64(mix64(tok + 0x632be59bd9b4e019ull) ^ (uint64_t)off);
}

// Walk the tree in evaluation order (as apply_composite does) and count each
// product; a composite child whose product was seen before is not walked
// again (its evaluation will come from the cache).
static void plan_walk(const isvd_operator *op, uint64_t tok, bool transpose, std::vector<std::pair<uint64_t, int>> &cnt) {
  auto visit = [&](const isvd_operator *c, uint64_t in) {
    const uint64_t k = product_key(c, in, transpose);
    for (auto &e : cnt)
      if (e.first == k) {
        ++e.second;
        return k;
      }
    cnt.emplace_back(k, 1);
    if (c->compose >= 0) plan_walk(c, in, transpose, cnt);
    return k;
  };
  const int m = (int)op->child.size();
  const bool summing = op->compose == ISVD_COMPOSE_SUM || (op->compose == ISVD_COMPOSE_HCAT && !transpose) ||
                       (op->compose == ISVD_COMPOSE_VCAT && transpose);
  if (op->compose == ISVD_COMPOSE_PRODUCT) {
    uint64_t cur = tok;
    for (int step = 0; step < m; ++step) cur = visit(op->child[transpose ? step : m - 1 - step], cur);
    return;
  }
  int64_t off = 0;
  for (int i = 0; i < m; ++i) {
    const isvd_operator *c = op->child[i];
    const uint64_t in = summing && op->compose != ISVD_COMPOSE_SUM ? slice_token(tok, off) : tok;
    visit(c, in);
    off += op->compose == ISVD_COMPOSE_HCAT ? c->cols : c->rows;
  }
}

void plan_product_cache(isvd_operator *op) {
  for (int t = 0; t < 2; ++t) {
    std::vector<std::pair<uint64_t, int>> cnt;
    plan_walk(op, 1, t == 1, cnt);
    op->cache_keys[t].clear();
    for (const auto &e : cnt)
      if (e.second > 1) op->cache_keys[t].push_back(e.first);
  }
}

// The cache of one evaluation: slot i holds the product with token keys[i]
// once done[i].
struct ProductCache {
  const std::vector<uint64_t> *keys = nullptr;
  char *base = nullptr;
  size_t slot_bytes = 0;
  bool done[ISVD_MAX_CHILDREN * 8] = {};
  int find(uint64_t k) const {
    if (!keys) return -1;
    for (size_t i = 0; i < keys->size() && i < sizeof done; ++i)
      if ((*keys)[i] == k) return (int)i;
    return -1;
  }
};

// Products of a composite node from its children's (Sec. 4, App. A.3):
//   (sum_i w_i M_i) G = sum_i w_i (M_i G), and likewise for the transpose;
//   [M_1 | ...] G = sum_i M_i G_i (G_i: the rows of G meeting M_i's columns),
//   [M_1 | ...]^T H = [M_1^T H ; ...];  [M_1 ; ...] G = [M_1 G ; ...],
//   [M_1 ; ...]^T H = sum_i M_i^T H_i;  (M_1 ... M_m) G = M_1 (... (M_m G)),
//   (M_1 ... M_m)^T H = M_m^T (... (M_1^T H)).
// Children run one after another on the stream and share one scratch region;
// sums accumulate into `out` through one block pass per extra child.  A
// product that the tree forms more than once (the same child on the same
// input, e.g. N G inside N^2 + N, or N^T H in [N | N^2]^T H) is formed once
// into a cache slot and read from there afterwards (the lazy cache of App.
// A.3, keyed by the chain of operators applied to the input).
static isvd_status apply_composite(isvd_operator *op, const void *G, int64_t ldg, int32_t b, void *out, int64_t ldo,
                                   int dtype, bool transpose, const ApplyScratch &sc, cudaStream_t s,
                                   ProductCache *pc, uint64_t tok) {
  const size_t es = dtype_size(dtype);
  const int64_t ldz = round_up(b, 8);
  const int m = (int)op->child.size();
  ProductCache own;
  if (!pc) {  // the root of this evaluation
    own.keys = op->cache_on ? &op->cache_keys[transpose ? 1 : 0] : nullptr;
    own.base = sc.cache_base;
    own.slot_bytes = sc.cache_slot_bytes;
    pc = &own;
  }
  // child c on `in` (token in_tok): the product lands in `o` (ld ldoo), or in
  // its cache slot, whose address is returned in *res (ld ldz) -- then the
  // caller reads it from there
  auto child_apply = [&](isvd_operator *c, const void *in, int64_t ldi, uint64_t in_tok, void *o, int64_t ldoo,
                         const void **res, int64_t *ldres) -> isvd_status {
    const uint64_t key = product_key(c, in_tok, transpose);
    const int slot = pc->find(key);
    void *dst = o;
    int64_t ldd = ldoo;
    if (slot >= 0) {
      dst = pc->base + (size_t)slot * pc->slot_bytes;
      ldd = ldz;
    }
    if (slot < 0 || !pc->done[slot]) {
      ApplyScratch cs;
      apply_scratch_carve(c, b, dtype, transpose, sc.child_base, &cs);
      if (c->compose >= 0) ISVD_TRY(apply_composite(c, in, ldi, b, dst, ldd, dtype, transpose, cs, s, pc, in_tok));
      else ISVD_TRY(apply_impl(c, in, ldi, b, dst, ldd, dtype, transpose, cs, s));
      if (slot >= 0) pc->done[slot] = true;
    }
    *res = dst;
    *ldres = ldd;
    return ISVD_OK;
  };
  // out-of-place result into o (o = w x + [o])
  auto deliver = [&](const void *res, int64_t ldr, void *o, int64_t ldoo, int64_t rows, double w, bool first) {
    if (res == o && first && w == 1.0) return cudaSuccess;
    if (res == o && first) return axpy_launch(o, ldoo, o, ldoo, rows, b, w, true, dtype, s);
    return axpy_launch(res, ldr, o, ldoo, rows, b, w, first, dtype, s);
  };
  auto rows_at = [&](const void *p, int64_t ld, int64_t r0) { return (char *)p + (size_t)r0 * ld * es; };
  const int64_t rows_out = transpose ? op->cols : op->rows;
  const bool summing = op->compose == ISVD_COMPOSE_SUM || (op->compose == ISVD_COMPOSE_HCAT && !transpose) ||
                       (op->compose == ISVD_COMPOSE_VCAT && transpose);
  const void *res = nullptr;
  int64_t ldr = 0;
  if (summing) {
    int64_t off = 0;  // first row of G_i (concatenations)
    for (int i = 0; i < m; ++i) {
      isvd_operator *c = op->child[i];
      const bool whole = op->compose == ISVD_COMPOSE_SUM;
      const void *in = whole ? G : (const void *)rows_at(G, ldg, off);
      const uint64_t in_tok = whole ? tok : slice_token(tok, off);
      const double w = op->weight[i];
      ISVD_TRY(child_apply(c, in, ldg, in_tok, i == 0 ? out : sc.ct1, i == 0 ? ldo : ldz, &res, &ldr));
      ISVD_CUDA_TRY(deliver(res, ldr, out, ldo, rows_out, w, i == 0));
      off += op->compose == ISVD_COMPOSE_HCAT ? c->cols : c->rows;
    }
    return ISVD_OK;
  }
  if (op->compose == ISVD_COMPOSE_HCAT || op->compose == ISVD_COMPOSE_VCAT) {
    int64_t off = 0;  // first row of child i's block of out
    for (int i = 0; i < m; ++i) {
      isvd_operator *c = op->child[i];
      const int64_t crows = op->compose == ISVD_COMPOSE_HCAT ? c->cols : c->rows;
      void *o = rows_at(out, ldo, off);
      ISVD_TRY(child_apply(c, G, ldg, tok, o, ldo, &res, &ldr));
      ISVD_CUDA_TRY(deliver(res, ldr, o, ldo, crows, 1.0, true));
      off += crows;
    }
    return ISVD_OK;
  }
  // product: right to left (transpose: left to right), two temporaries in turn
  const void *cur = G;
  int64_t ldc = ldg;
  uint64_t cur_tok = tok;
  void *tmp[2] = {sc.ct1, sc.ct2};
  int which = 0;
  for (int step = 0; step < m; ++step) {
    isvd_operator *c = op->child[transpose ? step : m - 1 - step];
    const bool last = step == m - 1;
    // the temporary that does not hold the current input
    if (tmp[which] == cur) which ^= 1;
    void *dst = last ? out : tmp[which];
    ISVD_TRY(child_apply(c, cur, ldc, cur_tok, dst, last ? ldo : ldz, &res, &ldr));
    if (last) ISVD_CUDA_TRY(deliver(res, ldr, out, ldo, rows_out, 1.0, true));
    cur = res;
    ldc = ldr;
    cur_tok = product_key(c, cur_tok, transpose);
    which ^= 1;
  }
  return ISVD_OK;
}

uint64_t tree_generation(const isvd_operator *op) {
  uint64_t g = op->generation * 0x9E3779B97F4A7C15ull + op->serial;
  for (const isvd_operator *c : op->child) g = (g * 1000003ull) ^ tree_generation(c);
  return g;
}

// With a row gather S: (S M) G = S (M G) and (S M)^T H = M^T (S^T H).
isvd_status apply_impl(isvd_operator *op, const void *G, int64_t ldg, int32_t b, void *out, int64_t ldo, int dtype,
                       bool transpose, const ApplyScratch &sc, cudaStream_t s) {
  if (op->compose >= 0) return apply_composite(op, G, ldg, b, out, ldo, dtype, transpose, sc, s, nullptr, 1);
  const isvd_operator_desc &d = op->desc;
  if (!d.gather_rows) return apply_form(op, G, ldg, b, out, ldo, dtype, transpose, sc, s);
  const int64_t ldz = round_up(b, 8);
  if (!transpose) {
    ISVD_TRY(apply_form(op, G, ldg, b, sc.gz, ldz, dtype, false, sc, s));
    ISVD_CUDA_TRY(gather_launch(sc.gz, ldz, d.gather_rows, d.n_gather, b, out, ldo, false, dtype, s));
    return ISVD_OK;
  }
  ISVD_CUDA_TRY(cudaMemsetAsync(sc.gz, 0, dtype_size(dtype) * (size_t)op->n * ldz, s));
  ISVD_CUDA_TRY(gather_launch(G, ldg, d.gather_rows, d.n_gather, b, sc.gz, ldz, true, dtype, s));
  return apply_form(op, sc.gz, ldz, b, out, ldo, dtype, true, sc, s);
}

}  // namespace isvd

using namespace isvd;

static std::atomic<uint64_t> g_next_serial{1};  // operator serials, unique in the process

extern "C" {

const char *isvd_last_error(void) { return isvd::last_error(); }

const char *isvd_status_string(isvd_status s) {
  switch (s) {
    case ISVD_OK: return "ok";
    case ISVD_ERR_INVALID_ARGUMENT: return "invalid argument";
    case ISVD_ERR_INVALID_GRAPH: return "invalid graph";
    case ISVD_ERR_SHAPE: return "shape mismatch";
    case ISVD_ERR_NOT_POSITIVE_DEFINITE: return "Gram matrix not positive definite";
    case ISVD_ERR_TIMEOUT: return "device wait timed out";
    case ISVD_ERR_WORKSPACE: return "workspace allocation failed";
    case ISVD_ERR_CUDA: return "CUDA error";
    case ISVD_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

isvd_status isvd_create_operator(const isvd_operator_desc *desc, const isvd_allocator *alloc, void *stream,
                                 isvd_operator **out) {
  if (!desc || !out) return fail(ISVD_ERR_INVALID_ARGUMENT, "null descriptor or output");
  *out = nullptr;
  isvd_operator *op = new isvd_operator();
  op->serial = g_next_serial.fetch_add(1);
  op->desc = *desc;
  if (alloc) {
    if (!alloc->alloc || !alloc->free) {
      delete op;
      return fail(ISVD_ERR_INVALID_ARGUMENT, "allocator with null callbacks");
    }
    op->alloc = *alloc;
    op->has_alloc = true;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const isvd_status st = create_impl(desc, op, s);
  if (st != ISVD_OK) {
    const std::string keep = isvd::last_error();
    cudaStreamSynchronize(s);
    cudaGetLastError();
    isvd_destroy_operator(op);
    isvd::set_error("%s", keep.c_str());
    return st;
  }
  // descriptor copies must not keep pointers into caller-owned host arrays
  op->desc.coeffs = nullptr;
  op->desc.lr_alpha = nullptr;
  *out = op;
  return ISVD_OK;
}

isvd_status isvd_compose_operators(isvd_compose kind, isvd_operator *const *ops, int32_t count,
                                   const double *weights, const isvd_allocator *alloc, void *stream,
                                   isvd_operator **out) {
  if (!ops || !out) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  *out = nullptr;
  if (kind < ISVD_COMPOSE_SUM || kind > ISVD_COMPOSE_PRODUCT)
    return fail(ISVD_ERR_INVALID_ARGUMENT, "unknown composite kind %d", (int)kind);
  if (count < 1 || count > ISVD_MAX_CHILDREN)
    return fail(ISVD_ERR_INVALID_ARGUMENT, "count must be in 1..%d", ISVD_MAX_CHILDREN);
  if (weights && kind != ISVD_COMPOSE_SUM) return fail(ISVD_ERR_INVALID_ARGUMENT, "weights are for SUM nodes only");
  if (alloc && (!alloc->alloc || !alloc->free)) return fail(ISVD_ERR_INVALID_ARGUMENT, "allocator with null callbacks");
  for (int i = 0; i < count; ++i) {
    if (!ops[i]) return fail(ISVD_ERR_INVALID_ARGUMENT, "null operator %d", i);
    if (weights && !std::isfinite(weights[i])) return fail(ISVD_ERR_INVALID_ARGUMENT, "weight %d is not finite", i);
  }
  int64_t rows = ops[0]->rows, cols = ops[0]->cols;
  for (int i = 1; i < count; ++i) {
    const isvd_operator *c = ops[i];
    switch (kind) {
      case ISVD_COMPOSE_SUM:
        if (c->rows != rows || c->cols != cols) return fail(ISVD_ERR_SHAPE, "SUM: operator %d has another shape", i);
        break;
      case ISVD_COMPOSE_HCAT:
        if (c->rows != rows) return fail(ISVD_ERR_SHAPE, "HCAT: operator %d has another row count", i);
        cols += c->cols;
        break;
      case ISVD_COMPOSE_VCAT:
        if (c->cols != cols) return fail(ISVD_ERR_SHAPE, "VCAT: operator %d has another column count", i);
        rows += c->rows;
        break;
      case ISVD_COMPOSE_PRODUCT:
        if (ops[i - 1]->cols != c->rows)
          return fail(ISVD_ERR_SHAPE, "PRODUCT: operator %d has %lld columns, operator %d %lld rows", i - 1,
                      (long long)ops[i - 1]->cols, i, (long long)c->rows);
        cols = c->cols;
        break;
    }
  }
  isvd_operator *op = new isvd_operator();
  op->serial = g_next_serial.fetch_add(1);
  op->compose = (int32_t)kind;
  op->child.assign(ops, ops + count);
  op->weight = weights ? std::vector<double>(weights, weights + count) : std::vector<double>(count, 1.0);
  op->rows = rows;
  op->cols = cols;
  plan_product_cache(op);
  if (alloc) {
    op->alloc = *alloc;
    op->has_alloc = true;
  }
  (void)stream;
  const cudaError_t e = cudaStreamCreateWithFlags(&op->capture_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    op->capture_stream = nullptr;
    isvd_destroy_operator(op);
    return fail(ISVD_ERR_CUDA, "stream creation failed: %s", cudaGetErrorString(e));
  }
  *out = op;
  return ISVD_OK;
}

isvd_status isvd_composite_cache(isvd_operator *op, int32_t enable) {
  if (!op) return fail(ISVD_ERR_INVALID_ARGUMENT, "null operator");
  if (op->compose < 0) return fail(ISVD_ERR_INVALID_ARGUMENT, "the product cache belongs to composite operators");
  op->cache_on = enable ? 1 : 0;
  invalidate_graphs(op);
  return ISVD_OK;
}

void isvd_destroy_operator(isvd_operator *op) {
  if (!op) return;
  cudaDeviceSynchronize();
  invalidate_graphs(op);
  batched_forget(op->serial);
  cudaStream_t s = nullptr;
  op_free(op, op->arena, s);
  for (void *p : op->owned) op_free(op, p, s);
  free_heavy(op, &op->heavy_A, s);
  free_heavy(op, &op->heavy_X, s);
  free_heavy(op, &op->heavy_XT, s);
  free_chunks(op, &op->chunk_A, s);
  free_chunks(op, &op->chunk_X, s);
  free_chunks(op, &op->chunk_XT, s);
  free_slab_plan(op, &op->slab_A, s);
  if (op->capture_stream) cudaStreamDestroy(op->capture_stream);
  if (op->side.fork) cudaEventDestroy(op->side.fork);
  if (op->side.join) cudaEventDestroy(op->side.join);
  if (op->side.stream) cudaStreamDestroy(op->side.stream);
  cudaStreamSynchronize(s);
  delete op;
}

isvd_status isvd_operator_shape(const isvd_operator *op, int64_t *rows, int64_t *cols) {
  if (!op || !rows || !cols) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  *rows = op->rows;
  *cols = op->cols;
  return ISVD_OK;
}

static isvd_status apply_entry(isvd_operator *op, const void *G, int64_t ldg, int32_t b, void *out, int64_t ldo,
                               isvd_dtype dtype, void *stream, bool transpose) {
  if (!op || !G || !out) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  if (dtype != ISVD_F32 && dtype != ISVD_BF16) return fail(ISVD_ERR_INVALID_ARGUMENT, "unknown dtype");
  if (b < 1 || b > 1024) return fail(ISVD_ERR_INVALID_ARGUMENT, "block width b must be in 1..1024");
  if (ldg < b || ldo < b || ldg % 8 || ldo % 8) return fail(ISVD_ERR_INVALID_ARGUMENT, "ld must be >= b and a multiple of 8");
  if (((uintptr_t)G | (uintptr_t)out) & 15) return fail(ISVD_ERR_INVALID_ARGUMENT, "blocks must be 16-byte aligned");
  const int dt = dtype == ISVD_F32 ? DT_F32 : DT_BF16;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = apply_scratch_bytes(op, b, dt, transpose);
  ISVD_TRY(ensure_arena(op, bytes, s));
  ApplyScratch sc;
  apply_scratch_carve(op, b, dt, transpose, (char *)op->arena, &sc);
  return apply_impl(op, G, ldg, b, out, ldo, dt, transpose, sc, s);
}

isvd_status isvd_apply(isvd_operator *op, const void *G, int64_t ldg, int32_t b, void *out, int64_t ldo,
                       isvd_dtype dtype, void *stream) {
  return apply_entry(op, G, ldg, b, out, ldo, dtype, stream, false);
}

isvd_status isvd_apply_T(isvd_operator *op, const void *G, int64_t ldg, int32_t b, void *out, int64_t ldo,
                         isvd_dtype dtype, void *stream) {
  return apply_entry(op, G, ldg, b, out, ldo, dtype, stream, true);
}

isvd_status isvd_get_tuning(const isvd_operator *op, isvd_tuning *out) {
  if (!op || !out) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  out->slab_cols_f32 = op->slab_cols_f32;
  out->slab_cols_bf16 = op->slab_cols_bf16;
  out->heavy_threshold = op->heavy_A.threshold;
  out->heavy_chunk = op->heavy_A.chunk;
  out->flags = (op->cache_hints ? ISVD_TUNE_CACHE_HINTS : 0) | (op->spmm_algo == 0 ? ISVD_TUNE_ROW_KERNEL : 0) |
               (op->spmm_algo == 3 ? ISVD_TUNE_SLAB_KERNEL : 0) |
               (op->spmm_algo == 2 ? ISVD_TUNE_RING_KERNEL : 0) | (op->hot_tags ? ISVD_TUNE_HOT_TAGS : 0) |
               (op->rows_occupancy >= 3 ? ISVD_TUNE_ROWS_OCC3 : 0) | (op->prefetch ? ISVD_TUNE_PREFETCH : 0) |
               (op->packed_temps ? ISVD_TUNE_PACKED : 0);
  out->chunk_nnz = op->chunk_nnz;
  out->l2_budget_mb = (int32_t)(op->tags_A.l2_budget >> 20);
  return ISVD_OK;
}

isvd_status isvd_set_tuning(isvd_operator *op, const isvd_tuning *t, void *stream) {
  if (!op || !t) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  if (op->compose >= 0) return fail(ISVD_ERR_UNSUPPORTED, "a composite operator has no launch shapes: tune its children");
  if (t->slab_cols_f32 < 4 || t->slab_cols_f32 > 256 || t->slab_cols_f32 % 4 || t->slab_cols_bf16 < 8 ||
      t->slab_cols_bf16 > 512 || t->slab_cols_bf16 % 8 || t->heavy_threshold < 32 || t->heavy_chunk < 32 ||
      t->chunk_nnz < 32 || t->chunk_nnz > (1 << 20) || t->l2_budget_mb < 1 || t->l2_budget_mb > 1024)
    return fail(ISVD_ERR_INVALID_ARGUMENT, "tuning field out of range");
  cudaStream_t s = (cudaStream_t)stream;
  ISVD_CUDA_TRY(cudaStreamSynchronize(s));
  invalidate_graphs(op);
  op->slab_cols_f32 = t->slab_cols_f32;
  op->slab_cols_bf16 = t->slab_cols_bf16;
  op->cache_hints = (t->flags & ISVD_TUNE_CACHE_HINTS) ? 1 : 0;
  op->spmm_algo = (t->flags & ISVD_TUNE_SLAB_KERNEL)  ? 3
                  : (t->flags & ISVD_TUNE_RING_KERNEL) ? 2
                  : (t->flags & ISVD_TUNE_ROW_KERNEL)  ? 0
                                                       : 1;
  op->hot_tags = (t->flags & ISVD_TUNE_HOT_TAGS) ? 1 : 0;
  op->rows_occupancy = (t->flags & ISVD_TUNE_ROWS_OCC3) ? 3 : 2;
  op->prefetch = (t->flags & ISVD_TUNE_PREFETCH) ? 1 : 0;
  op->packed_temps = (t->flags & ISVD_TUNE_PACKED) ? 1 : 0;
  op->chunk_nnz = t->chunk_nnz;
  op->tags_A.l2_budget = (int64_t)t->l2_budget_mb << 20;
  HeavyPlan *plans[3] = {&op->heavy_A, &op->heavy_X, &op->heavy_XT};
  for (HeavyPlan *hp : plans) {
    hp->threshold = t->heavy_threshold;
    hp->chunk = t->heavy_chunk;
  }
  ISVD_TRY(build_heavy(op, op->desc.A.rowptr, op->n, &op->heavy_A, s));
  ISVD_TRY(build_chunks(op, op->desc.A.rowptr, op->n, op->desc.A.nnz, &op->chunk_A, s));
  ISVD_TRY(build_slab_plan(op, op->desc.A.rowptr, op->n, op->heavy_A.threshold, op->heavy_A.chunk, &op->slab_A, s));
  if (op->desc.form == ISVD_FORM_CONCAT) {
    ISVD_TRY(build_heavy(op, op->x_rowptr, op->n, &op->heavy_X, s));
    ISVD_TRY(build_heavy(op, op->xt_rowptr, op->desc.d, &op->heavy_XT, s));
    ISVD_TRY(build_chunks(op, op->x_rowptr, op->n, op->x_nnz, &op->chunk_X, s));
    ISVD_TRY(build_chunks(op, op->xt_rowptr, op->desc.d, op->x_nnz, &op->chunk_XT, s));
  }
  return ISVD_OK;
}

}  // extern "C"
