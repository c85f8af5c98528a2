// Internal declarations shared by the libisvd translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

#include "isvd.h"

namespace isvd {

// ---- errors -----------------------------------------------------------------
void set_error(const char *fmt, ...);
isvd_status fail(isvd_status s, const char *fmt, ...);
const char *last_error();

#define ISVD_CUDA_TRY(expr)                                                                      \
  do {                                                                                           \
    cudaError_t e_ = (expr);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return ::isvd::fail(ISVD_ERR_CUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), \
                          __FILE__, __LINE__);                                                   \
  } while (0)

#define ISVD_TRY(expr)                   \
  do {                                   \
    isvd_status s_ = (expr);             \
    if (s_ != ISVD_OK) return s_;        \
  } while (0)

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
inline int64_t ceil_div(int64_t x, int64_t m) { return (x + m - 1) / m; }

constexpr int kNumSMs = 152;

// ---- dtype helpers ------------------------------------------------------------
enum DType : int { DT_F32 = 0, DT_BF16 = 1 };
inline size_t dtype_size(int dt) { return dt == DT_F32 ? 4 : 2; }

// ---- sparse products ---------------------------------------------------------
// One column slab of an SpMM: columns [col0, col0 + width) of the logical
// block, read from `in` and written to `out` (both already offset to the
// slab's first column and to the slab's row segment).  `group` lanes cooperate
// on one row (power of two, 1..32); each lane owns 16 bytes of columns.
struct SpmmSlab {
  const void *in;
  int64_t ldi;
  void *out;
  int64_t ldo;
  const void *axpy;  // optional, same layout as out (offset to the slab)
  int64_t lda;
  int32_t col0;      // first column of the slab in the low-rank coefficient block
  int32_t width;     // valid columns in this slab
  int32_t group;     // lanes per row
  int32_t hot_bucket;  // with column tags: gathers of columns in degree buckets >= this keep L2 priority
};

constexpr int kMaxSlabs = 24;

struct SpmmArgs {
  int64_t rows;
  const int32_t *rowptr;
  const int32_t *colidx;
  const float *values;      // nullable: all ones
  const float *colw;        // nullable: gathered weight of the source row j
  int32_t self_term;        // add colw_i * in_i (or in_i)
  const float *rowscale;    // nullable
  float scalar;             // multiplies the gathered sum
  float ax_scalar;          // axpy term: ax_scalar * ax_rowscale_i * axpy_i
  const float *ax_rowscale; // nullable
  int32_t lr_rank;          // low-rank epilogue: sum_t lr_alpha_t * u_it * c_t
  int32_t lr_ones_first;    // term 0 has u = 1; terms t >= 1 read lr_u column t-1
  const float *lr_u;        // nullable = ones; rows x (lr_rank - lr_ones_first) (ld lr_ldu)
  int64_t lr_ldu;
  const float *lr_c;        // lr_rank x lr_ldc (FP32)
  int64_t lr_ldc;
  float lr_alpha[ISVD_MAX_LOWRANK];
  int32_t heavy_threshold;  // rows with more nonzeros go through the split path
  int32_t cache_hints;      // L2 eviction-priority hints on gathers and streams
  const int32_t *tagged;    // nullable: colidx with degree buckets (RingTags), for the hints
  int32_t rows_occupancy;   // row kernel: 3 = compiled for 6 resident CTAs per SM (40 registers), else default
  int32_t prefetch;         // row kernel: L2 prefetch of the next row's first neighbour rows
  const int32_t *row_order; // nullable: rows by degree, largest first (narrow slabs visit rows in this order)
  int32_t nslabs;
  SpmmSlab slab[kMaxSlabs];
};

// Heavy rows: nonzeros split into chunks processed independently, partial
// sums combined in chunk order (deterministic).
struct HeavyPlan {
  int32_t n_rows = 0;       // heavy rows
  int32_t n_big = 0;        // the first n_big rows have more than kBigHubChunks chunks
  int32_t n_chunks = 0;
  int2 *chunks = nullptr;   // (row, first nnz) per chunk; chunk end = next chunk or row end
  int32_t *chunk_end = nullptr;
  int4 *rows = nullptr;     // (row, first chunk, chunk count, 0)
  int32_t threshold = 128;
  int32_t chunk = 128;
};

// Heavy rows with more chunks than this are summed by a whole CTA (eight
// warps over the chunks) instead of one warp.
constexpr int32_t kBigHubChunks = 32;

// Launch the SpMM described by `a` (dtype of in/axpy/out), splitting heavy
// rows per `hp` using `partial` (hp.n_chunks x pw FP32, pw >= slab columns).
// A second stream (and a fork / join event pair) on which the split hub rows
// run beside the row-group kernel; all null: one stream.
struct SideStream {
  cudaStream_t stream = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
cudaError_t spmm_launch(const SpmmArgs &a, int dtype, const HeavyPlan &hp, float *partial,
                        int64_t pw, cudaStream_t s, const SideStream &side);

// Column slabs for a block of width b (row-major, 16-byte aligned).
int make_slabs(int dtype, int32_t b, int32_t slab_cols, SpmmSlab *out);

// Packed-slab form: one launch per column slab over a work list of
// segments sorted by length, longest first: whole rows of at most `chunk`
// nonzeros (rows without nonzeros included, so that their epilogue runs) and
// the `chunk`-nonzero pieces of longer (hub) rows.  A hub piece stores its
// partial sum in its slot; the group that completes a hub's last piece adds
// the hub's partials in slot order and applies the epilogue, so results do
// not depend on the order in which pieces finish.
struct SlabPlan {
  int32_t n_items = 0;
  int4 *items = nullptr;        // (row, first nonzero, end, slot): slot -1 = a whole row
  int32_t n_hubs = 0;
  int4 *hubs = nullptr;         // (row, first slot, piece count, 0)
  int32_t *slot_hub = nullptr;  // hub of each slot
  int32_t n_slots = 0;
  int32_t *counters = nullptr;  // pieces finished per hub in the running launch (0 between launches)
  int32_t chunk = 128;
};
// partial: p.n_slots x pw FP32 (pw >= the widest slab).
cudaError_t spmm_slab_launch(const SpmmArgs &a, int dtype, const SlabPlan &p, float *partial, int64_t pw,
                             cudaStream_t s);

// Nonzero-balanced form: warps take chunks of CH consecutive nonzeros; rows
// crossing chunk boundaries (split) and rows without nonzeros (empty) are
// finished by two small passes.  row_of[e] is the row of nonzero e.
struct ChunkPlan {
  int64_t nnz = 0;
  int32_t CH = 512;
  int64_t nchunks = 0;
  int32_t *row_of = nullptr;
  int4 *split = nullptr;  // (row, first chunk, last chunk, 0)
  int32_t nsplit = 0;
  int32_t *empty = nullptr;
  int32_t nempty = 0;
};
// part: nchunks x 2 x pw FP32 partial sums (head / tail row of each chunk).
cudaError_t spmm_chunk_launch(const SpmmArgs &a, int dtype, const ChunkPlan &cp, float *part, int64_t pw,
                              cudaStream_t s);
int chunk_slab_cols(int dtype);

// Ring form (spmm_ring.cu): the same chunk plan, full-width gathers streamed
// through shared memory with cp.async.  One slab per launch (a.nslabs == 1)
// of at most ring_max_cols(dtype) columns.  Column tags: colidx with the
// column's degree bucket floor(log2 deg) in bits 26..30 (n < 2^26), and the
// number of columns per bucket; gathers of the hottest buckets whose rows fit
// l2_budget bytes get the L2 evict_last policy.
constexpr size_t kRingSmemBudget = 200 * 1024;
constexpr int64_t kRingL2Budget = 64ll << 20;
struct RingTags {
  const int32_t *tagged = nullptr;
  const int32_t *row_order = nullptr;  // rows of A by degree, largest first (ties in row order)
  int64_t hist[32] = {};
  int64_t l2_budget = 0;
};
int ring_max_cols(int dtype);
cudaError_t spmm_ring_launch(const SpmmArgs &a, int dtype, const ChunkPlan &cp, const RingTags &tags, float *part,
                             int64_t pw, cudaStream_t s);

// ---- dense helpers -----------------------------------------------------------
cudaError_t gaussian_launch(uint64_t seed, int64_t rows, int32_t cols, void *out, int64_t ld, int dtype,
                            cudaStream_t s);
cudaError_t philox_words_launch(uint64_t seed, int64_t rows, uint32_t *out, cudaStream_t s);

// c (r x b, FP32, ld ldc) = V^T G.  Column t of V is all ones when t == 0 and
// ones_first, or when V is null; otherwise column t - ones_first of V (rows x ldv).
cudaError_t lowrank_project_launch(const void *G, int64_t ldg, int dtype, int64_t rows, int32_t b,
                                   const float *V, int64_t ldv, int32_t r, int32_t ones_first,
                                   double *partial, int32_t n_part, float *c, int64_t ldc, cudaStream_t s);
int32_t lowrank_partials(int64_t rows);

// Gram W (FP64, l x l) = Q^T Q over rows; partial workspace n_part x l x l FP64.
// gate: when non-null and *gate_flag says so, the kernels return at once
// (conditional CholeskyQR passes).
struct PassGate {
  const int32_t *state = nullptr;  // orthonormalisation state (see small.cu)
  int32_t pass = 0;                // 1-based pass number; passes > 2 are conditional
};
int32_t gram_partials(int64_t rows);
cudaError_t gram_launch(const void *Q, int64_t ldq, int dtype, int64_t rows, int32_t l, double *partial,
                        int32_t n_part, double *W, PassGate g, cudaStream_t s);

// Q <- Q B in place on the tensor cores, B (l x l, FP32) upper triangular.
// colsum (nullable): FP64 partial column sums of the stored Q, one row of l
// per slot, gemm_colsum_parts(rows) slots (the all-ones projection of the
// product that reads Q next); colsum_reduce_launch sums them in a fixed order.
cudaError_t gemm_tri_inplace_launch(void *Q, int64_t ldq, int dtype, int64_t rows, int32_t l, const float *B,
                                    int64_t ldb, PassGate g, cudaStream_t s, double *colsum = nullptr);
int32_t gemm_colsum_parts(int64_t rows);
cudaError_t colsum_reduce_launch(const double *partial, int32_t parts, int32_t ld, int32_t b, int32_t ldc, float *out,
                                 cudaStream_t s);
// Out[:, 0:w] = Q B[:, 0:w] on the tensor cores (3xTF32), Q rows x l FP32, or
// with `subtract` Out[:, 0:w] -= Q B[:, 0:w] (Out must not overlap the columns
// of Q); *launched = false (nothing enqueued) where the layout does not suit it.
cudaError_t gemm_tc_launch(const float *Q, int64_t ldq, int64_t rows, int32_t l, const float *B, int64_t ldb,
                           int32_t w, float *out, int64_t ldo, bool *launched, cudaStream_t s,
                           bool subtract = false);

// out (rows x w) = Q (rows x l) B (l x w, FP32, ld ldb); upper: B upper
// triangular.  out may equal Q (in place) when w == l and out dtype == in dtype.
cudaError_t gemm_small_launch(const void *Q, int64_t ldq, int in_dtype, int64_t rows, int32_t l,
                              const float *B, int64_t ldb, int32_t w, bool upper, void *out,
                              int64_t ldo, int out_dtype, PassGate g, cudaStream_t s);

// W (c x m) = V S^+ (U^T Y) (Thm. 1).  partial: nparts x k x m FP64; Z: k x m FP32.
int32_t closed_form_parts(int64_t rows, int32_t k, int32_t m);
cudaError_t closed_form_launch(const float *U, int64_t ldu, const float *S, const float *V, int64_t ldv, int64_t r,
                               int64_t c, int32_t k, const float *Y, int64_t ldy, int32_t m, double rcond,
                               float *W, int64_t ldw, double *partial, int32_t nparts, float *Z, cudaStream_t s);

// out = X diag(S)^1/2 (Sec. 3.1 embeddings; out may equal X) and
// out[p] = <L_src[p], R_dst[p]> with range-checked indices (closed_form.cu).
cudaError_t embed_launch(const float *X, int64_t ldx, int64_t rows, int32_t k, const float *S, float *out,
                         int64_t ldo, cudaStream_t s);
cudaError_t pair_scores_launch(const float *L, int64_t ldl, int64_t rows, const float *R, int64_t ldr, int64_t cols,
                               int32_t k, const int32_t *src, const int32_t *dst, int64_t n_pairs, float *out,
                               isvd_info *info, cudaStream_t s);

// C (p x q, FP64 partials per row part: [parts][p][q]) = A^T B over `rows`
// rows on the tensor cores (gram_ab_tc.cu), p <= 128, q <= 160, A and B FP32
// with 16-byte aligned bases and rows; *launched = false (nothing enqueued)
// otherwise.  err (nullable, device int32): set to 1 when a bounded wait
// gave up.  gram_ab_parts: the partial count it uses for `rows` rows.
int32_t gram_ab_parts(int64_t rows);
cudaError_t gram_ab_launch(const float *A, int64_t lda, int32_t p, const float *B, int64_t ldb, int32_t q,
                           int64_t rows, double *partial, int32_t parts, int32_t *err, bool *launched,
                           cudaStream_t s);

// C (p x q, FP64 partials per row part) = A^T B over `rows` rows (closed_form.cu).
int32_t tn_tiles(int32_t p, int32_t q);
cudaError_t tn_partial_launch(const float *A, int64_t lda, const float *B, int64_t ldb, int64_t rows, int32_t p,
                              int32_t q, double *partial, int32_t nparts, cudaStream_t s);

// Dense X in the CONCAT operator (xdense.cu): P = X [G_0 | ... | G_L] and
// out_l = X^T P_l (P_0 = H copied into segment 0).  Scratch: xdense_scratch_bytes.
int32_t xdense_parts(int64_t n, int32_t d, int32_t q);
size_t xdense_scratch_bytes(int32_t d, int32_t segs, int32_t bseg, int64_t n);
cudaError_t xdense_forward(const float *X, int64_t n, int32_t d, const void *G, int64_t ldg, int dtype, int32_t b,
                           int32_t bseg, int32_t segs, void *P, int64_t ldp, void *scratch, cudaStream_t s);
cudaError_t xdense_transpose(const float *X, int64_t n, int32_t d, const float *H, int64_t ldh, int32_t b,
                             int32_t bseg, int32_t segs, float *P, int64_t ldp, float *out, int64_t ldo, void *scratch,
                             cudaStream_t s);

// ---- small FP64 kernels -------------------------------------------------------
// Orthonormalisation state block (device, int32[8]):
//  [0] last pass that needed a shift (0 = none)   [1] breakdown flag
constexpr int kOrthStateInts = 8;
cudaError_t orth_reset_launch(int32_t *state, cudaStream_t s);
// Cholesky of W (+ adaptive shift) -> Rinv (FP32, l x ldr), R (FP64 l x l, optional),
// accumulates Racc <- R Racc when Racc non-null.
cudaError_t chol_inv_launch(const double *W, int32_t l, int64_t rows, int dtype, float *Rinv, int64_t ldr,
                            double *R, double *Racc, double *tmp, int32_t *state, isvd_info *info, int32_t pass,
                            cudaStream_t s);
cudaError_t racc_init_launch(double *Racc, int32_t l, cudaStream_t s);
// The same step spread over a thread-block cluster (chol_cluster.cu); the
// cluster size it can use (16, 8, or 1 when none fits).
int chol_cluster_size();
cudaError_t chol_cluster_launch(const double *W, int32_t l, double u, float *Rinv, int64_t ldr, double *R,
                                double *Racc, double *tmp, int32_t *state, isvd_info *info, int32_t pass,
                                cudaStream_t s);
// SVD A = Uo diag(S) Vo^T of an l x l FP64 matrix by one-sided Jacobi on the
// columns of A^T.  Optional FP32 copies of the first k columns (Uk, Vk: l x k)
// and of S (k).  work: small_svd_work_doubles(l) FP64.
cudaError_t small_svd_launch(const double *A, int32_t l, double *Uo, double *S, double *Vo, double *work,
                             float *Uk, float *Vk, float *Sk, int32_t k, isvd_info *info, int32_t iters,
                             cudaStream_t s);
size_t small_svd_work_doubles(int32_t l);
cudaError_t small_kernels_init();
cudaError_t dense_kernels_init();

// Device buffers of one orthonormalisation (CholeskyQR2 with shift).
struct OrthBufs {
  double *gram_partial = nullptr;  // n_part x l x l FP64
  double *W = nullptr, *tmp = nullptr;  // l x l FP64 each
  float *Rinv = nullptr;          // l x l FP32
  int32_t *state = nullptr;       // kOrthStateInts
  int32_t n_part = 0;
  double *colsum = nullptr;       // nullable: gemm_colsum_parts(rows) x l column-sum partials of the result
};
isvd_status orth_enqueue(void *Q, int64_t ldq, int dt, int64_t rows, int32_t l, double *Racc, const OrthBufs &o,
                         isvd_info *info, cudaStream_t s);
// FP32 blocks of ISVD_MAX_BLOCK < l <= ISVD_MAX_BLOCK_WIDE columns (orth_wide.cu):
// 128-column panels by block Gram-Schmidt (two projections) and CholeskyQR2.
// o: buffers for 128 columns; wbuf: wide_orth_bytes(rows, l), 256-byte aligned.
size_t wide_orth_bytes(int64_t rows, int32_t l);
isvd_status wide_orth_enqueue(float *Q, int64_t ldq, int64_t rows, int32_t l, double *Racc, const OrthBufs &o,
                              char *wbuf, isvd_info *info, cudaStream_t s);

}  // namespace isvd

// ---- the operator ------------------------------------------------------------
struct isvd_operator {
  isvd_operator_desc desc{};
  isvd_allocator alloc{};
  bool has_alloc = false;
  int64_t n = 0, rows = 0, cols = 0;
  std::vector<double> coeffs;
  std::vector<double> lr_alpha;
  // device arrays owned by the operator
  float *deg = nullptr, *inv_d = nullptr, *s = nullptr, *s2 = nullptr;
  // X^T (CONCAT) and dense-X-as-CSR
  int32_t *xt_rowptr = nullptr, *xt_colidx = nullptr;
  float *xt_values = nullptr;
  int32_t *xd_rowptr = nullptr, *xd_colidx = nullptr;  // dense X viewed as CSR
  const int32_t *x_rowptr = nullptr, *x_colidx = nullptr;
  const float *x_values = nullptr;
  int64_t x_nnz = 0;
  isvd::HeavyPlan heavy_A, heavy_X, heavy_XT;
  isvd::ChunkPlan chunk_A, chunk_X, chunk_XT;
  isvd::SlabPlan slab_A;    // packed-slab work list of A
  isvd::RingTags tags_A;    // degree-bucket tags of A's columns (ring form)
  int32_t spmm_algo = 3;    // 0: row groups with hub splitting, 1: nonzero chunks, 2: ring, 3: packed slabs
  int32_t chunk_nnz = 512;
  std::vector<void *> owned;  // allocations released at destroy
  // workspace arena (grow only)
  void *arena = nullptr;
  size_t arena_bytes = 0;
  cudaStream_t capture_stream = nullptr;
  isvd::SideStream side;        // second stream: split hub rows beside the row-group kernel
  int32_t slab_cols_f32 = 64, slab_cols_bf16 = 128;
  int32_t cache_hints = 1;
  int32_t hot_tags = 1;     // row kernel: L2 priority only for gathers of hub columns
  int32_t rows_occupancy = 3;
  int32_t prefetch = 0;
  int32_t packed_temps = 0; // Horner temporaries stored slab by slab (each slab a dense [n][w] block)
  struct GraphEntry {
    uint64_t key[16];
    cudaGraphExec_t exec;
    int64_t kernel_nodes;
  };
  std::vector<GraphEntry> graphs;
  int64_t last_kernel_nodes = -1;
  uint64_t serial = 0;      // unique per operator in the process
  uint64_t generation = 0;  // bumped whenever captured graphs become stale
  // composite node (Sec. 4): compose >= 0 is an isvd_compose kind over the
  // referenced children; -1 is a leaf described by desc
  int32_t compose = -1;
  std::vector<isvd_operator *> child;
  std::vector<double> weight;
  // lazy product cache (App. A.3): the products (a child applied to a given
  // input) that one evaluation of this tree forms more than once, per
  // direction [transpose], each with a slot of the apply scratch; planned at
  // composition from the tree's structure
  std::vector<uint64_t> cache_keys[2];
  int32_t cache_on = 1;
};

namespace isvd {
void *op_alloc(isvd_operator *op, size_t bytes, cudaStream_t s);
void free_heavy(isvd_operator *op, HeavyPlan *hp, cudaStream_t s);
void free_chunks(isvd_operator *op, ChunkPlan *cp, cudaStream_t s);
void free_slab_plan(isvd_operator *op, SlabPlan *sp, cudaStream_t s);
void op_free(isvd_operator *op, void *p, cudaStream_t s);
isvd_status ensure_arena(isvd_operator *op, size_t bytes, cudaStream_t s);
// Drop the operator's captured graphs (workspace moved or launch shapes changed).
void invalidate_graphs(isvd_operator *op);
// Drop batched graphs that include the operator with this serial.
void batched_forget(uint64_t serial);

// Scratch layout for one apply (offsets into a region of the arena).
struct ApplyScratch {
  void *z1 = nullptr, *z2 = nullptr, *p = nullptr;  // Horner temps, CONCAT P block
  float *lr_c = nullptr;
  double *lr_partial = nullptr;
  // column sums of the input block already formed (by the orthonormalisation
  // that wrote it): the all-ones projection reduces them instead of reading
  // the block; ones_parts slots of ones_ld doubles
  const double *ones_parts = nullptr;
  int32_t ones_nparts = 0, ones_ld = 0;
  float *heavy_partial = nullptr;
  void *xdense = nullptr;  // dense-X products (CONCAT with dense X)
  void *gz = nullptr;      // row gather: the full-height product (n x b)
  // composite nodes: two block temporaries and the children's scratch
  void *ct1 = nullptr, *ct2 = nullptr;
  char *child_base = nullptr;
  // root composite: the lazy product cache's slots
  char *cache_base = nullptr;
  size_t cache_slot_bytes = 0;
};
// Generation of an operator and everything below it (composite graphs go
// stale when a child's workspace or launch shapes change).
uint64_t tree_generation(const isvd_operator *op);
size_t apply_scratch_bytes(const isvd_operator *op, int32_t b, int dtype, bool transpose);
void apply_scratch_carve(const isvd_operator *op, int32_t b, int dtype, bool transpose, char *base,
                         ApplyScratch *sc);
isvd_status apply_impl(isvd_operator *op, const void *G, int64_t ldg, int32_t b, void *out, int64_t ldo,
                       int dtype, bool transpose, const ApplyScratch &sc, cudaStream_t s);
}  // namespace isvd
