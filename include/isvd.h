/*
 * isvd.h -- C ABI of libisvd.so: randomized truncated SVD of an implicit
 * design matrix on one GB300 (sm_103a).
 *
 * Method: "Implicit SVD for Graph Representation Learning" (arXiv 2111.06312).
 *   - The matrix M is never formed.  Only M.G and M^T.G are evaluated from
 *     M's defining expression (Sec. 4 and App. A.3: shape, dot, T).
 *   - Two expression forms are supported:
 *       POLY:   M = sum_{k=1..K} c_k N^k + alpha 1 1^T + beta A + sum_t a_t u_t v_t^T
 *               (Eq. 3 is c_q from the context window, alpha = -lambda,
 *               beta = +lambda; Sec. 3.1 also allows N = Â)
 *       CONCAT: M = [X | N X | ... | N^L X]                       (Eq. 6)
 *     with N = T = D^-1 A (ISVD_NORM_ROW) or
 *          N = Â = (D+I)^-1/2 (A+I) (D+I)^-1/2 (ISVD_NORM_SYM_SELFLOOP)  (Sec. 2).
 *   - isvd_svd runs Alg. 1 (randomized range finder with power iterations,
 *     App. A.2) with orthonorm = CholeskyQR (Alg. 2, right), applied twice
 *     with an adaptive shift on breakdown, and Rayleigh-Ritz.
 *
 * Conventions (every entry point):
 *   - Pointers are DEVICE pointers unless marked HOST.
 *   - Dense blocks are row-major [rows][ld] with ld >= cols, ld % 8 == 0 and
 *     the base 16-byte aligned.  Columns at or beyond the logical width are
 *     never written by isvd_apply / isvd_apply_T.
 *   - The caller owns every buffer passed in.  An operator BORROWS the CSR
 *     and feature arrays of its descriptor for its whole lifetime.
 *   - Work is asynchronous on the given cudaStream_t (passed as void*; NULL is
 *     the legacy default stream).  isvd_create_operator synchronises once to
 *     validate its input.  Calls on one operator must be ordered (one stream,
 *     or explicit events): the operator owns a reusable workspace.
 *   - One device per process: kernel attributes (shared-memory sizes,
 *     cluster shapes) are set once per process, on the device current at the
 *     first call into the library.
 *   - Errors are returned as isvd_status; no exception or abort crosses the
 *     ABI.  isvd_last_error() returns a thread-local detail string.  Errors
 *     that only the GPU can see (CholeskyQR breakdown) are written to a
 *     device-resident isvd_info that the caller reads after synchronising.
 */
#ifndef ISVD_H_
#define ISVD_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ISVD_API __attribute__((visibility("default")))
#else
#define ISVD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ISVD_OK = 0,
  ISVD_ERR_INVALID_ARGUMENT = 1,   /* null pointer, bad ld/alignment, k < 1, ... */
  ISVD_ERR_INVALID_GRAPH = 2,      /* CSR not well formed, zero degree for T, asymmetric A */
  ISVD_ERR_SHAPE = 3,              /* block width or rank does not fit the operator */
  ISVD_ERR_NOT_POSITIVE_DEFINITE = 4, /* CholeskyQR broke down even with a shift */
  ISVD_ERR_TIMEOUT = 5,            /* a bounded device wait expired */
  ISVD_ERR_WORKSPACE = 6,          /* the allocator returned NULL */
  ISVD_ERR_CUDA = 7,               /* a CUDA runtime call failed (detail in last_error) */
  ISVD_ERR_UNSUPPORTED = 8         /* valid request outside what this library implements */
} isvd_status;

typedef enum { ISVD_F32 = 0, ISVD_BF16 = 1 } isvd_dtype;

/* FP32: all blocks stored in FP32, FP32-accurate Gram and products.
 * MIXED: power iterations store blocks in BF16 (FP32 accumulation), then one
 * FP32 refinement power step and an FP32 Rayleigh-Ritz.                     */
typedef enum { ISVD_PREC_FP32 = 0, ISVD_PREC_MIXED = 1 } isvd_precision;

typedef enum {
  ISVD_NORM_ROW = 0,          /* N = T = D^-1 A                   (Sec. 2) */
  ISVD_NORM_SYM_SELFLOOP = 1, /* N = Â = (D+I)^-1/2 (A+I) (D+I)^-1/2  (Sec. 2) */
  ISVD_NORM_SYM_NOSELF = 2    /* N = Â - (D+I)^-1 = (D+I)^-1/2 A (D+I)^-1/2: label
                                 re-use's adjacency, zero diagonal on a graph
                                 without self-loops (Sec. 5.3)                  */
} isvd_norm;

typedef enum {
  ISVD_FORM_POLY = 0,    /* sum_k c_k N^k + corrections         (Eq. 3) */
  ISVD_FORM_CONCAT = 1   /* [X | N X | ... | N^L X]             (Eq. 6) */
} isvd_form;

/* Sparse matrix in CSR: rowptr[rows+1] (rowptr[0] == 0, nondecreasing,
 * rowptr[rows] == nnz), colidx[nnz] in [0, cols), values[nnz] or NULL for a
 * pattern whose entries are all 1.  int32 indices: nnz < 2^31.             */
typedef struct {
  int64_t rows, cols, nnz;
  const int32_t *rowptr;
  const int32_t *colidx;
  const float *values;
} isvd_csr;

/* Workspace allocator.  alloc(bytes, stream, ctx) returns device memory that
 * is usable in stream order on `stream`, or NULL; free(ptr, stream, ctx)
 * releases it.  Pass NULL for the allocator to use cudaMallocAsync /
 * cudaFreeAsync.                                                            */
typedef struct {
  void *(*alloc)(size_t bytes, void *stream, void *ctx);
  void (*free)(void *ptr, void *stream, void *ctx);
  void *ctx;
} isvd_allocator;

enum {
  ISVD_FLAG_SKIP_SYMMETRY_CHECK = 1  /* trust that A is symmetric (pattern and values) */
};

#define ISVD_MAX_DEGREE 16
#define ISVD_MAX_LOWRANK 8
#define ISVD_MAX_BLOCK 160   /* largest block width l = k + p of isvd_svd (any precision) */
#define ISVD_MAX_BLOCK_WIDE 512  /* largest FP32 block width of isvd_svd, isvd_orthonormalize */

typedef struct {
  isvd_form form;
  isvd_norm norm;
  isvd_csr A;              /* n x n adjacency, both directions stored; symmetric */
  /* POLY */
  int32_t degree;          /* K in 1..ISVD_MAX_DEGREE */
  const double *coeffs;    /* HOST, c_1..c_K (copied at creation) */
  double ones_coeff;       /* alpha of alpha 1 1^T (Eq. 3: -lambda); 0 = none */
  double adj_coeff;        /* beta of beta A (Eq. 3 as printed: +lambda); 0 = none */
  int32_t lr_rank;         /* extra sum_t a_t u_t v_t^T terms, 0..ISVD_MAX_LOWRANK */
  const float *lr_u;       /* n x lr_rank row-major (ld = lr_rank) */
  const float *lr_v;       /* n x lr_rank row-major (ld = lr_rank) */
  const double *lr_alpha;  /* HOST, lr_rank values (copied) */
  /* CONCAT */
  int64_t d;               /* feature width */
  int32_t L;               /* propagation depth, >= 0 */
  isvd_csr X;              /* sparse X (n x d), or all-null when X_dense is given */
  const float *X_dense;    /* dense X, row-major n x d (ld = d) */
  int32_t flags;           /* ISVD_FLAG_* */
  /* Row gather (either form): the operator is M[gather_rows, :], the rows a
   * closed-form fit uses (Thm. 1 on the training rows).  DEVICE int32,
   * n_gather strictly increasing indices in [0, n); NULL = all rows. */
  const int32_t *gather_rows;
  int64_t n_gather;
} isvd_operator_desc;

/* Device-resident status of isvd_svd / isvd_orthonormalize, written by the
 * GPU.  status: an isvd_status.  chol_shifts: CholeskyQR passes that needed
 * a diagonal shift.  cholqr_passes: passes run.  iters_done: power
 * iterations completed.                                                      */
typedef struct {
  int32_t status;
  int32_t chol_shifts;
  int32_t cholqr_passes;
  int32_t iters_done;
} isvd_info;

typedef struct isvd_operator isvd_operator;

/* Build an operator from a descriptor (the leaf and symbolic nodes of
 * Sec. 4 / App. A.3 folded into one description).  Validates the CSR (and,
 * unless ISVD_FLAG_SKIP_SYMMETRY_CHECK, the symmetry of A) on the GPU,
 * computes degrees and scale vectors, builds X^T for CONCAT and the row
 * work lists of the sparse products.  Synchronises `stream` once.
 * Errors: INVALID_ARGUMENT, INVALID_GRAPH, UNSUPPORTED, WORKSPACE, CUDA.
 * On success *out owns device workspace; free with isvd_destroy_operator. */
ISVD_API isvd_status isvd_create_operator(const isvd_operator_desc *desc, const isvd_allocator *alloc,
                                 void *stream, isvd_operator **out);

/* Free an operator and its workspace (after its last stream work).  NULL ok. */
ISVD_API void isvd_destroy_operator(isvd_operator *op);

/* (rows, cols) of M: (n, n) for POLY, (n, d (L+1)) for CONCAT (App. A.3:
 * shape); rows = n_gather with a row gather. */
ISVD_API isvd_status isvd_operator_shape(const isvd_operator *op, int64_t *rows, int64_t *cols);

/* out (rows x b) = M G, G (cols x b): App. A.3 `dot`.  dtype gives the
 * storage type of G and out (FP32 accumulation either way).  G and out must
 * not overlap.  b in 1..1024. */
ISVD_API isvd_status isvd_apply(isvd_operator *op, const void *G, int64_t ldg, int32_t b, void *out,
                       int64_t ldo, isvd_dtype dtype, void *stream);

/* out (cols x b) = M^T G, G (rows x b): App. A.3 `T().dot`. */
ISVD_API isvd_status isvd_apply_T(isvd_operator *op, const void *G, int64_t ldg, int32_t b, void *out,
                         int64_t ldo, isvd_dtype dtype, void *stream);

/* Rank-k SVD of M by Alg. 1 with block width l = k + oversample (the paper
 * uses l = 2k), `iters` power iterations (Alg. 1's `iterations`), start block
 * N(0,1) from Philox4x32-10 keyed by `seed`.  Outputs: U (rows x k, ldu),
 * S (k, descending), V (cols x k, ldv), all FP32.  dev_info may be NULL.
 * Requires 1 <= k, l <= min(rows, cols) and l <= ISVD_MAX_BLOCK, or, in
 * ISVD_PREC_FP32, l <= ISVD_MAX_BLOCK_WIDE (the paper's l = 2k at ranks up
 * to 256): blocks wider than ISVD_MAX_BLOCK are orthonormalised in panels of
 * 128 columns (block Gram-Schmidt with two projections, then CholeskyQR2 per
 * panel), which gives the same thin QR up to rounding.  The sequence is
 * captured once per argument set into a CUDA graph and replayed.  Errors:
 * UNSUPPORTED (l > ISVD_MAX_BLOCK_WIDE, or l > ISVD_MAX_BLOCK in
 * ISVD_PREC_MIXED). */
ISVD_API isvd_status isvd_svd(isvd_operator *op, int32_t k, int32_t oversample, int32_t iters, uint64_t seed,
                     isvd_precision precision, float *U, int64_t ldu, float *S, float *V, int64_t ldv,
                     isvd_info *dev_info, void *stream);

/* Many independent rank-k SVDs (Alg. 1 on each problem) in one call: one
 * CUDA graph whose parallel branches run the problems side by side, so that
 * small problems together fill the GPU.  The paper has no batched form; each
 * problem's result equals that of isvd_svd with the same arguments.
 *   ops[i]   : distinct operators (each owns the workspace its problem uses);
 *   k[i]     : rank of problem i (HOST array); oversample and iters shared;
 *   seed + i : start-block seed of problem i;
 *   U[i], S[i], V[i] : HOST arrays of DEVICE pointers; U[i] is rows_i x k[i]
 *              and V[i] cols_i x k[i], dense (ld = k[i]); S[i] has k[i] values;
 *   dev_info : NULL or a DEVICE array of `count` isvd_info, one per problem.
 * The graph is captured on the first call with a given argument set and
 * replayed afterwards (the same operators, pointers and sizes).  Inside a
 * caller's stream capture the branches are forked into that capture.
 * Errors: INVALID_ARGUMENT (null, repeated operator, k < 1), SHAPE,
 * UNSUPPORTED (k + oversample > ISVD_MAX_BLOCK), WORKSPACE, CUDA. */
ISVD_API isvd_status isvd_svd_batched(isvd_operator *const *ops, const int32_t *k, int32_t count,
                                      int32_t oversample, int32_t iters, uint64_t seed, isvd_precision precision,
                                      float *const *U, float *const *S, float *const *V, isvd_info *dev_info,
                                      void *stream);

/* Kernel launches in the graph replayed by this thread's last
 * isvd_svd_batched call (-1 if none).  Introspection for benchmarks. */
ISVD_API int64_t isvd_batched_kernel_nodes(void);

/* The same batch in ONE persistent kernel (FP32): each problem is taken by
 * a team of 1..32 CTAs (one per rows_per_member rows, at most max_team) that
 * runs the whole of Alg. 1 for it, its members meeting at a per-problem stage counter
 * in device memory wherever a step reads rows another member wrote (the
 * sparse products, the summed Gram matrices and column sums).  Every wait is
 * bounded: one that runs out abandons that problem (status
 * ISVD_ERR_TIMEOUT in its isvd_info) and the kernel goes on with the others.
 * Arguments as isvd_svd_batched (precision FP32); results equal isvd_svd's up
 * to rounding.  Takes polynomial operators of an unweighted graph (Eq. 3 with
 * N = T or A-hat, at most the all-ones term; no values, beta A, low-rank
 * terms, row gather or composite nodes), k + oversample <=
 * ISVD_PERSISTENT_MAX_BLOCK, else ISVD_ERR_UNSUPPORTED.  opt may be NULL.
 * Workspace from each problem's operator (operator 0 also holds the queue).
 * Asynchronous on `stream`: one cooperative kernel launch after a few copies. */
#define ISVD_PERSISTENT_MAX_BLOCK 96
typedef struct {
  int32_t max_team;     /* CTAs per problem at most (0: 32) */
  int32_t rows_per_member; /* rows per team member (0: 16384) */
  int32_t spin_limit;   /* polls of a team wait before it gives up (0: ~4 million, seconds) */
  int32_t test_phantom; /* test only: every team waits for one member more than it has,
                           so that every wait runs out (the failure path, without a fault) */
} isvd_persistent_options;
ISVD_API isvd_status isvd_svd_batched_persistent(isvd_operator *const *ops, const int32_t *k, int32_t count,
                                                 int32_t oversample, int32_t iters, uint64_t seed,
                                                 float *const *U, float *const *S, float *const *V,
                                                 isvd_info *dev_info, const isvd_persistent_options *opt,
                                                 void *stream);

/* --- individual steps, exported for verification and reuse --------------- */

/* out[i][j] (rows x cols) = standard normal from Philox4x32-10 (Salmon et al.
 * 2011): counter (j/4, i mod 2^32, i / 2^32, 0), key (seed mod 2^32,
 * seed / 2^32), words (0,1) and (2,3) turned into normals j%4 = 0,1 and 2,3
 * by Box-Muller with u = (word + 1/2) 2^-32.  Alg. 1's start block.
 * dtype selects FP32 or BF16 storage.  Columns cols..ld-1 are set to zero. */
ISVD_API isvd_status isvd_gaussian(uint64_t seed, int64_t rows, int32_t cols, void *out, int64_t ld,
                          isvd_dtype dtype, void *stream);

/* Raw Philox4x32-10 words for counters (c0 = j, c1 = i mod 2^32,
 * c2 = i / 2^32, 0) with i in [0, rows), j in [0, 4): out[i][4 j + w]
 * (uint32, rows x 16).  For known-answer and bit-parity checks. */
ISVD_API isvd_status isvd_philox_words(uint64_t seed, int64_t rows, uint32_t *out, void *stream);

/* In-place orthonormalisation of Q (rows x l, FP32, ldq): CholeskyQR2
 * (Alg. 2, right, applied twice); when a Gram matrix is not numerically
 * positive definite a diagonal shift is added and two further plain passes
 * follow (up to 4 passes).  R_out (DEVICE, l x l FP64, row-major, upper)
 * receives R with Q_in = Q_out R, or NULL.  dev_info as in
 * isvd_svd.  Uses the operator's workspace (any operator; pass the one whose
 * calls this is ordered with).  l <= ISVD_MAX_BLOCK_WIDE (above
 * ISVD_MAX_BLOCK in 128-column panels, as in isvd_svd); ldq >= l and a
 * multiple of 8, Q 16-byte aligned (else ISVD_ERR_INVALID_ARGUMENT). */
ISVD_API isvd_status isvd_orthonormalize(isvd_operator *op, float *Q, int64_t rows, int32_t l, int64_t ldq,
                                double *R_out, isvd_info *dev_info, void *stream);

/* isvd_orthonormalize without any allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * when they need it (code running inside another framework's allocator or
 * memory-pool callback, latency-bound services that forbid cudaMalloc on the
 * hot path because it can synchronise the device).  Its scratch is one
 * file-scope device array of about 10 MB that every GPU which loads the
 * library holds until the process exits.
 *   - Same arguments and results as isvd_orthonormalize (no operator), but
 *     l <= ISVD_NOALLOC_MAX_BLOCK (64); larger l returns ISVD_ERR_UNSUPPORTED.
 *   - The first call on a device sets up that device: it looks up the
 *     array's device address, and loading the library's code for that device
 *     (the array itself and the kernels, on their first use) makes the CUDA
 *     driver allocate device memory.  Make that first call outside the
 *     no-allocation context, as a warm-up, and before any stream capture on
 *     that device; later calls allocate nothing.
 *   - Kernel attributes (shared-memory sizes, cluster shapes) are set once
 *     per process, on the device current at the first call into the
 *     library: use the library from one device per process.
 *   - Every call shares the one array: calls that overlap on the GPU (other
 *     streams, other host threads) race and corrupt each other's results.
 *     Order them on one stream.  dev_info NULL uses a slot in the array that
 *     is cleared at the start of each call.
 *   - Calls no cudaMalloc, cudaFree or allocating library routine. */
#define ISVD_NOALLOC_MAX_BLOCK 64
ISVD_API isvd_status isvd_orthonormalize_noalloc(float *Q, int64_t rows, int32_t l, int64_t ldq, double *R_out,
                                                 isvd_info *dev_info, void *stream);

/* Closed-form weights from a rank-k SVD of M (Sec. 3, Thm. 1): the least-norm
 * minimiser of ||M W - Y||_F is M^+ Y; with M ~ U diag(S) V^T it is
 *     W = V diag(S)^+ U^T Y.
 * All pointers DEVICE, FP32, row-major: U (r x k, ld ldu), S (k), V (c x k,
 * ld ldv), Y (r x m, ld ldy), W (c x m, ld ldw, written).  r x c is the
 * operator's shape.  Label matrices with zero rows outside the training set
 * fit zero targets there; a fit on the training rows alone takes the SVD of
 * the row-gathered operator instead.  diag(S)^+ inverts S_i > rcond * max(S) and zeroes
 * the rest.  U^T Y is summed in FP64 across row parts.  1 <= k, m <=
 * ISVD_MAX_BLOCK.  Workspace from the operator's allocator; asynchronous on
 * `stream`. */
ISVD_API isvd_status isvd_closed_form(isvd_operator *op, const float *U, int64_t ldu, const float *S, const float *V,
                                      int64_t ldv, int32_t k, const float *Y, int64_t ldy, int32_t m, double rcond,
                                      float *W, int64_t ldw, void *stream);

/* Composite nodes of the symbolic representation (Sec. 4, App. A.3):
 *   SUM      M = sum_i w_i M_i          (all children of one shape)
 *   HCAT     M = [M_1 | M_2 | ...]      (columns side by side; equal row counts)
 *   VCAT     M = [M_1 ; M_2 ; ...]      (rows stacked; equal column counts)
 *   PRODUCT  M = M_1 M_2 ... M_m        (cols(M_i) == rows(M_{i+1}))
 * Label re-use (Sec. 5.3) is HCAT(M_NC, PRODUCT(N0, [Y | N0 Y])) with N0 =
 * ISVD_NORM_SYM_NOSELF; pseudo-dropout is VCAT(M, PD(M)). */
typedef enum {
  ISVD_COMPOSE_SUM = 0,
  ISVD_COMPOSE_HCAT = 1,
  ISVD_COMPOSE_VCAT = 2,
  ISVD_COMPOSE_PRODUCT = 3
} isvd_compose;

#define ISVD_MAX_CHILDREN 16

/* Build a composite operator over `count` (1..ISVD_MAX_CHILDREN) existing
 * operators, leaves or composites.  The children are referenced, not
 * copied or owned: they must outlive the composite and keep their tuning
 * (a change of a child's tuning or workspace is picked up at the next call).
 * weights: HOST, SUM only (count values, finite; NULL = all ones); must be
 * NULL for the other kinds.  The result works with isvd_apply, isvd_apply_T,
 * isvd_svd, isvd_closed_form, isvd_orthonormalize; products are formed from
 * the children's products in child order (sums and accumulations of the
 * concatenations through one extra block pass each).  Not accepted by
 * isvd_svd_batched, isvd_set_tuning or isvd_autotune (UNSUPPORTED): tune the
 * children.  Errors: INVALID_ARGUMENT (null pointers, bad count or
 * weights), SHAPE (children that do not fit the kind), CUDA. */
ISVD_API isvd_status isvd_compose_operators(isvd_compose kind, isvd_operator *const *ops, int32_t count,
                                            const double *weights, const isvd_allocator *alloc, void *stream,
                                            isvd_operator **out);

/* Lazy product cache of a composite (App. A.3: intermediate products cached
 * by the chain of operators applied to the input).  At composition the tree
 * is walked in evaluation order and every product that one evaluation forms
 * more than once (the same child applied to the same input: N G inside
 * N^2 + N, N^T H inside [N | N^2]^T H, M G inside [M ; M]) gets a slot of
 * the apply workspace (rows x round8(b) elements each); a call then forms it
 * once and reads it from its slot afterwards.  The results are bit for bit
 * those of the uncached evaluation.  enable = 0 turns the cache off for this
 * composite (evaluated as the root of a call), 1 (the default) on; drops
 * captured graphs.  Errors: INVALID_ARGUMENT (null, or a leaf operator). */
ISVD_API isvd_status isvd_composite_cache(isvd_operator *op, int32_t enable);

/* Network-embedding outputs of a rank-k SVD (Sec. 3.1): the rows and columns
 * of M are embedded as L = U diag(S)^1/2 and R = V diag(S)^1/2, so that
 * L R^T = U diag(S) V^T.  One call scales one factor: out = X diag(S)^1/2.
 * DEVICE, FP32, row-major: X (rows x k, ld ldx), S (k, >= 0; a negative
 * entry gives NaN columns), out (rows x k, ld ldo).  out == X scales in place;
 * other overlaps are undefined.  rows == 0 is a no-op.  Asynchronous on
 * `stream`.  Errors: INVALID_ARGUMENT (null pointer, ld < k), SHAPE (k < 1). */
ISVD_API isvd_status isvd_embed(const float *X, int64_t ldx, int64_t rows, int32_t k, const float *S, float *out,
                                int64_t ldo, void *stream);

/* Similarity of the node at row i and the node at column j (Sec. 3.1):
 * f(i, j) = <L_i, R_j> = U_i^T diag(S) V_j, for each pair p:
 * out[p] = f(src[p], dst[p]).  DEVICE: L (rows x k, ld ldl), R (cols x k,
 * ld ldr) FP32 row-major; src, dst (n_pairs, int32); out (n_pairs, FP32).
 * Products in FP32 per lane, summed across the warp in FP64 in a fixed order
 * (bitwise reproducible).  A pair with src outside [0, rows) or dst outside
 * [0, cols) gets NaN and, if dev_info is not NULL, dev_info->status =
 * ISVD_ERR_INVALID_ARGUMENT (left unchanged otherwise).  n_pairs == 0 is a
 * no-op.  Asynchronous on `stream`. */
ISVD_API isvd_status isvd_pair_scores(const float *L, int64_t ldl, int64_t rows, const float *R, int64_t ldr,
                                      int64_t cols, int32_t k, const int32_t *src, const int32_t *dst,
                                      int64_t n_pairs, float *out, isvd_info *dev_info, void *stream);

/* Gaussian-kernel edge function (Sec. 5.1, App. A.4).  With U (rows x k),
 * S (k, >= 0) and V (cols x k) from a rank-k SVD, a pair (i, j) scores
 *     f(i, j) = U_i^T diag(w) V_j,   w_c = sum_x pi_x S_c^x,
 * x on the 301-point grid 0.5, 0.505, ..., 2.0 (the truncation interval
 * [0.5, 2]) and pi = softmax_x(-(x - mu)^2 exp(s_bar)), s_bar = log(1/(2 s^2)):
 * the expectation of S^x under N(mu, s) truncated to the interval.  mu = 1
 * with s -> 0 gives w = S (the plain SVD score).  All factors DEVICE, FP32,
 * row-major.  `work`: DEVICE scratch of isvd_edge_kernel_work_doubles(k)
 * doubles, owned by the caller; calls that share it must be ordered on one
 * stream.  Pairs out of range: NaN score (loss: NaN), and dev_info->status =
 * ISVD_ERR_INVALID_ARGUMENT when dev_info is not NULL.  Sums are in a fixed
 * order (bitwise repeatable).  Asynchronous on `stream`. */
ISVD_API int64_t isvd_edge_kernel_work_doubles(int32_t k);

/* w3 (DEVICE, 3k doubles, written) = [w | dw/dmu | dw/ds_bar], in FP64. */
ISVD_API isvd_status isvd_edge_kernel_weights(const float *S, int32_t k, double mu, double s_bar, double *w3,
                                              void *stream);

/* out[p] = f(src[p], dst[p]) (FP32), src in [0, rows), dst in [0, cols). */
ISVD_API isvd_status isvd_edge_kernel_scores(const float *U, int64_t ldu, int64_t rows, const float *V,
                                             int64_t ldv, int64_t cols, int32_t k, const float *S, double mu,
                                             double s_bar, const int32_t *src, const int32_t *dst, int64_t n_pairs,
                                             float *out, double *work, int64_t work_doubles, isvd_info *dev_info,
                                             void *stream);

/* Link-prediction objective of Eq. 9 over n_pos edges (pos_src[p], pos_dst[p])
 * and n_neg non-edges:  L = -mean_pos log sigma(f) - k_neg mean_neg
 * log(1 - sigma(f)), and its gradient.  out (DEVICE, 3 doubles, written) =
 * [L, dL/dmu, dL/ds_bar].  n_pos >= 1, n_neg >= 0, k_neg >= 0. */
ISVD_API isvd_status isvd_edge_kernel_loss(const float *U, int64_t ldu, int64_t rows, const float *V, int64_t ldv,
                                           int64_t cols, int32_t k, const float *S, double mu, double s_bar,
                                           const int32_t *pos_src, const int32_t *pos_dst, int64_t n_pos,
                                           const int32_t *neg_src, const int32_t *neg_dst, int64_t n_neg,
                                           double k_neg, double *out, double *work, int64_t work_doubles,
                                           isvd_info *dev_info, void *stream);

/* Split-ReLU layer of the fine-tuning network (Sec. 5.2):
 *     Z = [X Wp]_+ - [X Wn]_+        ([t]_+ = max(t, 0))
 * X (n x d, ld ldx), Wp and Wn (d x e, row-major, ld e), all DEVICE FP32;
 * 1 <= d, e <= ISVD_MAX_BLOCK.  The forward writes Z (n x e, ld ldz) and the
 * pre-activations Ap = X Wp, An = X Wn (n x e each, ld lda), which the
 * backward takes: with Gp = dZ * 1[Ap > 0] and Gn = -dZ * 1[An > 0],
 *     dWp = X^T Gp, dWn = X^T Gn (d x e, ld e, written),
 *     dX = Gp Wp^T + Gn Wn^T (n x d, ld lddx; dX NULL: not formed).
 * The dense products run on the tensor cores (3xTF32) where the blocks'
 * bases and row pitches are 16-byte aligned, on the CUDA cores otherwise;
 * X^T G is summed in FP64 across row ranges in a fixed order.  `work`: DEVICE
 * scratch of isvd_split_relu_work_bytes(n, d, e) bytes, 256-byte aligned,
 * owned by the caller.  Asynchronous on `stream`.  Errors: INVALID_ARGUMENT
 * (null pointer, leading dimension), SHAPE (d or e out of range), WORKSPACE
 * (work too small or misaligned), CUDA. */
ISVD_API size_t isvd_split_relu_work_bytes(int64_t n, int32_t d, int32_t e);
ISVD_API isvd_status isvd_split_relu_forward(const float *X, int64_t ldx, int64_t n, int32_t d, const float *Wp,
                                             const float *Wn, int32_t e, float *Z, int64_t ldz, float *Ap, float *An,
                                             int64_t lda, void *stream);
ISVD_API isvd_status isvd_split_relu_backward(const float *X, int64_t ldx, int64_t n, int32_t d, const float *Wp,
                                              const float *Wn, int32_t e, const float *Ap, const float *An,
                                              int64_t lda, const float *dZ, int64_t ldz, float *dX, int64_t lddx,
                                              float *dWp, float *dWn, void *work, size_t work_bytes, void *stream);

/* SVD of a small square upper-triangular-or-dense FP64 matrix by one-sided
 * Jacobi on its transpose (the Rayleigh-Ritz step of Alg. 1, done as
 * SVD(R^T) after a QR of B^T).  A (l x l, row-major, DEVICE) = Uo diag(S) Vo^T
 * with Uo, Vo (l x l, FP64, row-major) and S (l, FP64, descending).
 * 1 <= l <= ISVD_MAX_BLOCK_WIDE.  dev_info (nullable): status, and the
 * number of Jacobi sweeps run in iters_done (60 at most). */
ISVD_API isvd_status isvd_small_svd(isvd_operator *op, const double *A, int32_t l, double *Uo, double *S,
                           double *Vo, isvd_info *dev_info, void *stream);

/* Launch shape of the sparse products (no counterpart in the paper, which ran
 * library kernels).  slab_cols_*: columns of the dense block processed per
 * pass over the CSR (the gathered slab of the block should stay L2-resident);
 * heavy_threshold: rows with more nonzeros are split into chunks of
 * heavy_chunk nonzeros whose partial sums are combined in order.  Slabs
 * narrower than 32 lanes hold several rows per warp; their rows of A are
 * visited in degree order (largest first, fixed at operator construction). */
typedef struct {
  int32_t slab_cols_f32;   /* 4..256, multiple of 4 (above 128: two 16-byte chunks per lane) */
  int32_t slab_cols_bf16;  /* 8..512, multiple of 8 (above 256: two chunks per lane) */
  int32_t heavy_threshold; /* >= 32 */
  int32_t heavy_chunk;     /* >= 32 */
  int32_t flags;           /* ISVD_TUNE_* */
  int32_t chunk_nnz;       /* nonzeros per warp chunk of the balanced kernels, 32..2^20 */
  int32_t l2_budget_mb;    /* L2 megabytes granted to gathered hub rows (HOT_TAGS), 1..1024 */
} isvd_tuning;

/* The sparse-product kernel: ISVD_TUNE_ROW_KERNEL (row groups with hub
 * splitting), ISVD_TUNE_RING_KERNEL (nonzero chunks, full-width gathers
 * streamed through shared memory; takes precedence), neither: nonzero chunks
 * over narrow column slabs. */
enum {
  ISVD_TUNE_CACHE_HINTS = 1, /* L2 eviction priorities: keep gathered (hub) rows, stream the rest */
  ISVD_TUNE_ROW_KERNEL = 2,
  ISVD_TUNE_RING_KERNEL = 4,
  ISVD_TUNE_HOT_TAGS = 8,    /* with CACHE_HINTS: keep priority only for hub columns (by degree) */
  ISVD_TUNE_ROWS_OCC3 = 16,  /* row kernel compiled for high occupancy (FP32: 6 CTAs of 256 threads per SM, BF16: 5) */
  ISVD_TUNE_PREFETCH = 32,   /* row kernel: L2 prefetch of the next row's first neighbour rows */
  ISVD_TUNE_PACKED = 64,     /* polynomial form: the Horner iterates between two sparse products are
                                stored slab by slab, each column slab a dense [n][width] block, so
                                that a slab's gathered rows fill whole L2 lines */
  ISVD_TUNE_SLAB_KERNEL = 128 /* products with A: one launch per column slab over a length-sorted
                                 list of rows and hub pieces (hub partials summed in piece order by
                                 the group finishing the last piece); implies PACKED; takes
                                 precedence over the other kernels.  It always sets L2 policies
                                 (gathered slab rows evict_last, the CSR stream, the axpy operand
                                 and the output evict_first); CACHE_HINTS concerns the others */
};

/* Read / replace the operator's launch shapes.  isvd_set_tuning rebuilds the
 * row split lists (synchronises `stream`) and drops captured graphs.
 * Errors: INVALID_ARGUMENT (out-of-range field), WORKSPACE, CUDA. */
ISVD_API isvd_status isvd_get_tuning(const isvd_operator *op, isvd_tuning *out);
ISVD_API isvd_status isvd_set_tuning(isvd_operator *op, const isvd_tuning *t, void *stream);

/* Choose the operator's sparse-product launch shape for block width b and
 * storage dtype by timing isvd_apply for a fixed list of candidates (row
 * kernel: occupancy, L2 budget for hub columns, hub split threshold, wide
 * slabs; the ring kernel), keep the fastest (applied with isvd_set_tuning and
 * copied to *out when out is not NULL).  cache_path (HOST, may be NULL): a text
 * file of earlier results keyed by the operator's shape and degree histogram,
 * b, dtype and the device name; a hit applies the stored shape without timing,
 * a miss appends the new result.  Synchronises `stream`; allocates two probe
 * blocks through the operator's allocator.  No counterpart in the paper.
 * Errors: INVALID_ARGUMENT, WORKSPACE, CUDA (the previous shape is restored). */
ISVD_API isvd_status isvd_autotune(isvd_operator *op, int32_t b, isvd_dtype dtype, const char *cache_path,
                                   isvd_tuning *out, void *stream);

/* Failure-detection self-test: launches one CTA that waits, through the same
 * bounded mbarrier wait the tensor-core kernels use, on a barrier that nothing
 * arrives on; after spin_limit polls (1..2^24) the wait gives up and the kernel
 * sets dev_info->status to ISVD_ERR_TIMEOUT and returns, leaving the context
 * usable.  dev_info: DEVICE isvd_info, cleared by the caller.  No counterpart
 * in the paper. */
ISVD_API isvd_status isvd_selftest_wait(int32_t spin_limit, isvd_info *dev_info, void *stream);

/* Number of kernel launches in the CUDA graph that the last isvd_svd call on
 * this operator replayed (-1 if none yet).  Introspection for benchmarks. */
ISVD_API int64_t isvd_graph_kernel_nodes(const isvd_operator *op);

ISVD_API const char *isvd_status_string(isvd_status s);
ISVD_API const char *isvd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ISVD_H_ */
