/*
 * FP64 CPU oracle for the implicit randomized SVD of "Implicit SVD for Graph
 * Representation Learning" (arXiv 2111.06312).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or helper with the CUDA path; the two meet only through the seeded
 * inputs of the synthetic generators.
 *
 * Everything is plain, slow and in FP64: loops written from the definitions
 * in the paper, no blocking, no fusion, no reordering beyond what the
 * definitions state.  OpenMP parallelises independent output rows only.
 *
 * What is computed, and where it is defined:
 *   - T = D^-1 A and  Â = (D+I)^-1/2 (A+I) (D+I)^-1/2            (Sec. 2)
 *   - Â - (D+I)^-1, the adjacency of label re-use, whose diagonal is
 *     zero on a graph without self-loops                           (Sec. 5.3)
 *   - M_NE = sum_q c_q T^q - lambda (1 1^T - A)                    (Sec. 3.1, Eq. 3)
 *     with the all-ones and adjacency coefficients given separately, plus
 *     optional low-rank terms sum_t a_t u_t v_t^T (the outer-product leaves
 *     of Sec. 4)
 *   - M_NC = [X | ÂX | ... | Â^L X]                               (Sec. 3.2, Eq. 6)
 *   - products M G and M^T G from those expressions                (Sec. 4; App. A.3),
 *     also of a row selection M[rows, :] (the training rows of Thm. 1's fit)
 *   - composite nodes: weighted sums, side-by-side and stacked
 *     concatenations and products of operators                     (Sec. 4, App. A.3;
 *     label re-use and pseudo-dropout of Sec. 5.3 are built from them)
 *   - orthonormOurs: L = chol(Q^T Q), Q <- Q (L^-1)^T              (Alg. 2, right)
 *     applied twice (CholeskyQR2) with a shift on breakdown
 *   - orthonormHalko: Householder QR                               (Alg. 2, left)
 *   - iSVD, the randomized range finder with power iterations      (Alg. 1)
 *   - one-sided Jacobi SVD (Hestenes) for the small / explicit SVDs
 *   - Philox4x32-10 + Box-Muller for the N(0,1) start block        (Alg. 1; the
 *     generator is Salmon et al., SC 2011, which the paper leaves unspecified)
 *
 * Parity pins (tests/test_oracle_*.py) tie each function to something other
 * than itself: closed-form spectra, published Philox answers, LAPACK, exact
 * invariants.  No function here is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Operator description                                                      */
/* ------------------------------------------------------------------------ */

typedef struct orc_op_s {
  int32_t form;        /* 0: polynomial  sum_k c_k N^k ; 1: concatenation     */
  int32_t norm;        /* 0: N = T = D^-1 A ; 1: N = Â ; 2: N = Â - (D+I)^-1    */
  int64_t n;           /* nodes                                                */
  const int32_t *rowptr, *colidx; /* CSR of A (n x n)                          */
  const double *aval;  /* edge weights, NULL = all ones                        */
  int32_t degree;      /* K (polynomial)                                        */
  const double *coeff; /* c_1..c_K                                             */
  double ones_coeff;   /* alpha: adds alpha * 1 1^T  (Eq. 3 has -lambda)        */
  double adj_coeff;    /* beta:  adds beta  * A      (Eq. 3 has +lambda)        */
  int64_t d;           /* feature dimension (concatenation)                    */
  int32_t L;           /* number of propagation blocks (concatenation)          */
  const int32_t *xrowptr, *xcolidx; const double *xval; /* sparse X, or     */
  const double *xdense; /* dense X, row-major n x d                            */
  int32_t lr_rank;     /* extra terms sum_t a_t u_t v_t^T (polynomial form)     */
  const double *lr_u, *lr_v; /* n x lr_rank, row-major                         */
  const double *lr_alpha;
  const int32_t *grows; /* row gather M[grows, :] (the training rows of Thm. 1's
                           fit), NULL = all rows                             */
  int64_t ngather;
  /* Composite nodes of the symbolic representation (Sec. 4, App. A.3): kind
   * 0 is a leaf (the fields above); 1: sum_i w_i M_i ; 2: [M_1 | M_2 | ...]
   * (columns side by side, equal row counts) ; 3: [M_1 ; M_2 ; ...] (rows
   * stacked, equal column counts) ; 4: the product M_1 M_2 ... M_m.         */
  int32_t kind;
  int32_t nchild;
  const struct orc_op_s *const *child;
  const double *weight; /* kind 1: w_i, NULL = all ones                       */
} orc_op;

static double a_val(const orc_op *op, int64_t e) { return op->aval ? op->aval[e] : 1.0; }

/* d_i = sum_j A_ij (Sec. 2: D is the diagonal degree matrix) */
static void degrees(const orc_op *op, double *deg) {
  for (int64_t i = 0; i < op->n; ++i) {
    double s = 0.0;
    for (int64_t e = op->rowptr[i]; e < op->rowptr[i + 1]; ++e) s += a_val(op, e);
    deg[i] = s;
  }
}

static int64_t full_rows(const orc_op *op) { return op->n; }

int64_t orc_rows(const orc_op *op) {
  if (op->kind == 0) return op->grows ? op->ngather : full_rows(op);
  if (op->kind == 3) {
    int64_t r = 0;
    for (int i = 0; i < op->nchild; ++i) r += orc_rows(op->child[i]);
    return r;
  }
  return orc_rows(op->child[0]); /* sum, side by side, product: the first factor's rows */
}

int64_t orc_cols(const orc_op *op) {
  if (op->kind == 0) return op->form == 0 ? op->n : op->d * (op->L + 1);
  if (op->kind == 2) {
    int64_t c = 0;
    for (int i = 0; i < op->nchild; ++i) c += orc_cols(op->child[i]);
    return c;
  }
  if (op->kind == 4) return orc_cols(op->child[op->nchild - 1]);
  return orc_cols(op->child[0]);
}

/* ------------------------------------------------------------------------ */
/* Leaf products                                                             */
/* ------------------------------------------------------------------------ */

/* out = N P  (n x b).  N = T:  out_i = (1/d_i) sum_j A_ij P_j.
 * N = Â: out_i = sum_j (A+I)_ij P_j / sqrt((d_i+1)(d_j+1)).
 * N = Â - (D+I)^-1: the same without the identity term (norm 2).           */
static void norm_apply(const orc_op *op, const double *deg, const double *P, double *out, int64_t b) {
  const int64_t n = op->n;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) {
    double *o = out + i * b;
    for (int64_t c = 0; c < b; ++c) o[c] = 0.0;
    if (op->norm == 0) {
      for (int64_t e = op->rowptr[i]; e < op->rowptr[i + 1]; ++e) {
        const int64_t j = op->colidx[e];
        const double t = a_val(op, e) / deg[i];
        for (int64_t c = 0; c < b; ++c) o[c] += t * P[j * b + c];
      }
    } else {
      for (int64_t e = op->rowptr[i]; e < op->rowptr[i + 1]; ++e) {
        const int64_t j = op->colidx[e];
        const double t = a_val(op, e) / sqrt((deg[i] + 1.0) * (deg[j] + 1.0));
        for (int64_t c = 0; c < b; ++c) o[c] += t * P[j * b + c];
      }
      if (op->norm == 1) {
        const double t = 1.0 / (deg[i] + 1.0); /* the identity term, (I)_ii */
        for (int64_t c = 0; c < b; ++c) o[c] += t * P[i * b + c];
      }
    }
  }
}

/* out = N^T P, by the definition (N^T)_ji = N_ij: a scatter over the rows
 * of A.  No symmetry of A is assumed.  Serial (scatter).                      */
static void norm_apply_T(const orc_op *op, const double *deg, const double *P, double *out, int64_t b) {
  const int64_t n = op->n;
  memset(out, 0, sizeof(double) * n * b);
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t e = op->rowptr[i]; e < op->rowptr[i + 1]; ++e) {
      const int64_t j = op->colidx[e];
      const double t = op->norm == 0 ? a_val(op, e) / deg[i]
                                     : a_val(op, e) / sqrt((deg[i] + 1.0) * (deg[j] + 1.0));
      for (int64_t c = 0; c < b; ++c) out[j * b + c] += t * P[i * b + c];
    }
    if (op->norm == 1) {
      const double t = 1.0 / (deg[i] + 1.0);
      for (int64_t c = 0; c < b; ++c) out[i * b + c] += t * P[i * b + c];
    }
  }
}

/* out (+)= A P  or  A^T P  (scatter for the transpose) */
static void adj_apply_acc(const orc_op *op, const double *P, double *out, int64_t b, double beta, int transpose) {
  const int64_t n = op->n;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = op->rowptr[i]; e < op->rowptr[i + 1]; ++e) {
      const int64_t j = op->colidx[e];
      const double t = beta * a_val(op, e);
      if (!transpose)
        for (int64_t c = 0; c < b; ++c) out[i * b + c] += t * P[j * b + c];
      else
        for (int64_t c = 0; c < b; ++c) out[j * b + c] += t * P[i * b + c];
    }
}

/* out = X P (n x b) where P is d x b; ld of P is b. */
static void x_apply(const orc_op *op, const double *P, int64_t ldp, double *out, int64_t b) {
  const int64_t n = op->n, d = op->d;
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t i = 0; i < n; ++i) {
    double *o = out + i * b;
    for (int64_t c = 0; c < b; ++c) o[c] = 0.0;
    if (op->xdense) {
      for (int64_t f = 0; f < d; ++f) {
        const double x = op->xdense[i * d + f];
        for (int64_t c = 0; c < b; ++c) o[c] += x * P[f * ldp + c];
      }
    } else {
      for (int64_t e = op->xrowptr[i]; e < op->xrowptr[i + 1]; ++e) {
        const int64_t f = op->xcolidx[e];
        const double x = op->xval[e];
        for (int64_t c = 0; c < b; ++c) o[c] += x * P[f * ldp + c];
      }
    }
  }
}

/* out = X^T P (d x b), P n x b; out written with leading dimension ldo. */
static void x_apply_T(const orc_op *op, const double *P, double *out, int64_t ldo, int64_t b) {
  const int64_t n = op->n, d = op->d;
  for (int64_t f = 0; f < d; ++f)
    for (int64_t c = 0; c < b; ++c) out[f * ldo + c] = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (op->xdense) {
      for (int64_t f = 0; f < d; ++f) {
        const double x = op->xdense[i * d + f];
        for (int64_t c = 0; c < b; ++c) out[f * ldo + c] += x * P[i * b + c];
      }
    } else {
      for (int64_t e = op->xrowptr[i]; e < op->xrowptr[i + 1]; ++e) {
        const int64_t f = op->xcolidx[e];
        const double x = op->xval[e];
        for (int64_t c = 0; c < b; ++c) out[f * ldo + c] += x * P[i * b + c];
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Implicit products M G and M^T G (Sec. 4: only these are needed for SVD)   */
/* ------------------------------------------------------------------------ */

/* G is (cols x b), out is (rows x b), both row-major with ld = b (the full M). */
static int apply_full(const orc_op *op, const double *G, int64_t b, double *out, int transpose) {
  const int64_t n = op->n;
  double *deg = (double *)malloc(sizeof(double) * n);
  degrees(op, deg);
  if (op->form == 0) {
    /* sum_{k=1..K} c_k N^k G  (or (N^T)^k), powers formed one after another */
    double *P = (double *)malloc(sizeof(double) * n * b);
    double *Pn = (double *)malloc(sizeof(double) * n * b);
    memcpy(P, G, sizeof(double) * n * b);
    memset(out, 0, sizeof(double) * n * b);
    for (int k = 1; k <= op->degree; ++k) {
      if (!transpose) norm_apply(op, deg, P, Pn, b);
      else norm_apply_T(op, deg, P, Pn, b);
      double *t = P; P = Pn; Pn = t;
      const double ck = op->coeff[k - 1];
      for (int64_t x = 0; x < n * b; ++x) out[x] += ck * P[x];
    }
    /* alpha * 1 (1^T G): the all-ones matrix is symmetric */
    if (op->ones_coeff != 0.0) {
      for (int64_t c = 0; c < b; ++c) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += G[i * b + c];
        for (int64_t i = 0; i < n; ++i) out[i * b + c] += op->ones_coeff * s;
      }
    }
    if (op->adj_coeff != 0.0) adj_apply_acc(op, G, out, b, op->adj_coeff, transpose);
    /* sum_t a_t u_t (v_t^T G); the transpose swaps u and v */
    for (int t = 0; t < op->lr_rank; ++t) {
      const double *u = transpose ? op->lr_v : op->lr_u;
      const double *v = transpose ? op->lr_u : op->lr_v;
      for (int64_t c = 0; c < b; ++c) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += v[i * op->lr_rank + t] * G[i * b + c];
        for (int64_t i = 0; i < n; ++i) out[i * b + c] += op->lr_alpha[t] * u[i * op->lr_rank + t] * s;
      }
    }
    free(P);
    free(Pn);
  } else {
    /* M = [X | ÂX | ... | Â^L X], n x d(L+1); block l of G is rows l*d..(l+1)*d-1 */
    const int64_t d = op->d;
    const int L = op->L;
    double *P = (double *)malloc(sizeof(double) * n * b);
    double *Pn = (double *)malloc(sizeof(double) * n * b);
    if (!transpose) {
      /* M G = sum_l Â^l (X G_l) */
      memset(out, 0, sizeof(double) * n * b);
      for (int l = 0; l <= L; ++l) {
        x_apply(op, G + (int64_t)l * d * b, b, P, b);
        for (int s = 0; s < l; ++s) {
          norm_apply(op, deg, P, Pn, b);
          double *t = P; P = Pn; Pn = t;
        }
        for (int64_t x = 0; x < n * b; ++x) out[x] += P[x];
      }
    } else {
      /* block l of M^T G = (Â^l X)^T G = X^T (Â^T)^l G */
      memcpy(P, G, sizeof(double) * n * b);
      for (int l = 0; l <= L; ++l) {
        x_apply_T(op, P, out + (int64_t)l * d * b, b, b);
        if (l < L) {
          norm_apply_T(op, deg, P, Pn, b);
          double *t = P; P = Pn; Pn = t;
        }
      }
    }
    free(P);
    free(Pn);
  }
  free(deg);
  return 0;
}

static int composite_apply(const orc_op *op, const double *G, int64_t b, double *out, int transpose);

/* With a row gather S (rows grows of the identity): (S M) G = S (M G) and
 * (S M)^T H = M^T (S^T H), S^T H placing row i of H at row grows[i]. */
int orc_apply(const orc_op *op, const double *G, int64_t b, double *out, int transpose) {
  if (op->kind != 0) return composite_apply(op, G, b, out, transpose);
  if (!op->grows) return apply_full(op, G, b, out, transpose);
  const int64_t nf = full_rows(op);
  double *F = (double *)calloc((size_t)(nf * b), sizeof(double));
  int rc;
  if (!transpose) {
    rc = apply_full(op, G, b, F, 0);
    for (int64_t i = 0; i < op->ngather; ++i)
      for (int64_t c = 0; c < b; ++c) out[i * b + c] = F[op->grows[i] * b + c];
  } else {
    for (int64_t i = 0; i < op->ngather; ++i)
      for (int64_t c = 0; c < b; ++c) F[op->grows[i] * b + c] += G[i * b + c];
    rc = apply_full(op, F, b, out, 1);
  }
  free(F);
  return rc;
}

/* Products of a composite node from its children's products:
 *   (sum_i w_i M_i) G = sum_i w_i (M_i G), and the same for the transpose;
 *   [M_1 | ... | M_m] G = sum_i M_i G_i, G_i the rows of G that meet M_i's
 *     columns;  [M_1 | ... | M_m]^T H = [M_1^T H ; ... ; M_m^T H];
 *   [M_1 ; ... ; M_m] G = [M_1 G ; ... ; M_m G];  [M_1 ; ... ; M_m]^T H =
 *     sum_i M_i^T H_i, H_i the rows of H that meet M_i's rows;
 *   (M_1 ... M_m) G = M_1 (... (M_m G));  (M_1 ... M_m)^T H = M_m^T (... (M_1^T H)). */
static int composite_apply(const orc_op *op, const double *G, int64_t b, double *out, int transpose) {
  const int64_t rout = transpose ? orc_cols(op) : orc_rows(op);
  const int m = op->nchild;
  int rc = 0;
  if (op->kind == 1 || (op->kind == 2 && !transpose) || (op->kind == 3 && transpose)) {
    double *T = (double *)malloc(sizeof(double) * (rout > 0 ? rout : 1) * b);
    memset(out, 0, sizeof(double) * rout * b);
    int64_t off = 0; /* first row of G_i (side by side / stacked) */
    for (int i = 0; i < m; ++i) {
      const orc_op *ci = op->child[i];
      const double *Gi = op->kind == 1 ? G : G + off * b;
      rc |= orc_apply(ci, Gi, b, T, transpose);
      const double w = (op->kind == 1 && op->weight) ? op->weight[i] : 1.0;
      for (int64_t x = 0; x < rout * b; ++x) out[x] += w * T[x];
      off += op->kind == 2 ? orc_cols(ci) : orc_rows(ci);
    }
    free(T);
  } else if (op->kind == 2 || op->kind == 3) {
    int64_t off = 0; /* first row of child i's block of the output */
    for (int i = 0; i < m; ++i) {
      const orc_op *ci = op->child[i];
      rc |= orc_apply(ci, G, b, out + off * b, transpose);
      off += op->kind == 2 ? orc_cols(ci) : orc_rows(ci);
    }
  } else if (op->kind == 4) {
    const double *cur = G;
    double *prev = NULL;
    for (int step = 0; step < m; ++step) {
      const orc_op *ci = op->child[transpose ? step : m - 1 - step];
      const int64_t ro = transpose ? orc_cols(ci) : orc_rows(ci);
      double *dst = step == m - 1 ? out : (double *)malloc(sizeof(double) * (ro > 0 ? ro : 1) * b);
      rc |= orc_apply(ci, cur, b, dst, transpose);
      free(prev);
      prev = step == m - 1 ? NULL : dst;
      cur = dst;
    }
  } else {
    rc = -1;
  }
  return rc;
}

static int explicit_full(const orc_op *op, double *M);
int orc_explicit(const orc_op *op, double *M);

/* Dense composite: the children's dense matrices combined by the node's
 * definition (weighted sum, placement side by side or stacked, product). */
static int composite_explicit(const orc_op *op, double *M) {
  const int64_t r = orc_rows(op), c = orc_cols(op);
  const int m = op->nchild;
  int rc = 0;
  if (op->kind == 1) {
    memset(M, 0, sizeof(double) * r * c);
    double *E = (double *)malloc(sizeof(double) * r * c);
    for (int i = 0; i < m; ++i) {
      rc |= orc_explicit(op->child[i], E);
      const double w = op->weight ? op->weight[i] : 1.0;
      for (int64_t x = 0; x < r * c; ++x) M[x] += w * E[x];
    }
    free(E);
  } else if (op->kind == 2) {
    int64_t off = 0; /* first column of child i */
    for (int i = 0; i < m; ++i) {
      const int64_t ci = orc_cols(op->child[i]);
      double *E = (double *)malloc(sizeof(double) * r * ci);
      rc |= orc_explicit(op->child[i], E);
      for (int64_t a = 0; a < r; ++a)
        for (int64_t j = 0; j < ci; ++j) M[a * c + off + j] = E[a * ci + j];
      free(E);
      off += ci;
    }
  } else if (op->kind == 3) {
    int64_t off = 0; /* first row of child i */
    for (int i = 0; i < m; ++i) {
      rc |= orc_explicit(op->child[i], M + off * c);
      off += orc_rows(op->child[i]);
    }
  } else if (op->kind == 4) {
    /* P <- P E_i, left to right */
    int64_t pc = orc_cols(op->child[0]);
    double *P = (double *)malloc(sizeof(double) * r * pc);
    rc |= orc_explicit(op->child[0], P);
    for (int i = 1; i < m; ++i) {
      const int64_t ec = orc_cols(op->child[i]);
      double *E = (double *)malloc(sizeof(double) * pc * ec);
      rc |= orc_explicit(op->child[i], E);
      double *Pn = (double *)calloc((size_t)(r * ec), sizeof(double));
      for (int64_t a = 0; a < r; ++a)
        for (int64_t t = 0; t < pc; ++t)
          for (int64_t j = 0; j < ec; ++j) Pn[a * ec + j] += P[a * pc + t] * E[t * ec + j];
      free(E);
      free(P);
      P = Pn;
      pc = ec;
    }
    memcpy(M, P, sizeof(double) * r * c);
    free(P);
  } else {
    rc = -1;
  }
  return rc;
}

/* Dense M (rows x cols, row-major) built from its definition, tiny sizes. */
int orc_explicit(const orc_op *op, double *M) {
  if (op->kind != 0) return composite_explicit(op, M);
  if (!op->grows) return explicit_full(op, M);
  const int64_t nf = full_rows(op), c = orc_cols(op);
  double *F = (double *)malloc(sizeof(double) * nf * c);
  const int rc = explicit_full(op, F);
  for (int64_t i = 0; i < op->ngather; ++i) memcpy(M + i * c, F + op->grows[i] * c, sizeof(double) * c);
  free(F);
  return rc;
}

static int explicit_full(const orc_op *op, double *M) {
  const int64_t n = op->n;
  double *deg = (double *)malloc(sizeof(double) * n);
  degrees(op, deg);
  /* dense N */
  double *N = (double *)calloc((size_t)(n * n), sizeof(double));
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t e = op->rowptr[i]; e < op->rowptr[i + 1]; ++e) {
      const int64_t j = op->colidx[e];
      N[i * n + j] += op->norm == 0 ? a_val(op, e) / deg[i]
                                    : a_val(op, e) / sqrt((deg[i] + 1.0) * (deg[j] + 1.0));
    }
    if (op->norm == 1) N[i * n + i] += 1.0 / (deg[i] + 1.0);
  }
  if (op->form == 0) {
    double *P = (double *)calloc((size_t)(n * n), sizeof(double));
    double *Pn = (double *)calloc((size_t)(n * n), sizeof(double));
    for (int64_t i = 0; i < n; ++i) P[i * n + i] = 1.0;
    memset(M, 0, sizeof(double) * n * n);
    for (int k = 1; k <= op->degree; ++k) {
#pragma omp parallel for
      for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
          double s = 0.0;
          for (int64_t t = 0; t < n; ++t) s += N[i * n + t] * P[t * n + j];
          Pn[i * n + j] = s;
        }
      double *t = P; P = Pn; Pn = t;
      for (int64_t x = 0; x < n * n; ++x) M[x] += op->coeff[k - 1] * P[x];
    }
    for (int64_t x = 0; x < n * n; ++x) M[x] += op->ones_coeff;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t e = op->rowptr[i]; e < op->rowptr[i + 1]; ++e)
        M[i * n + op->colidx[e]] += op->adj_coeff * a_val(op, e);
    for (int t = 0; t < op->lr_rank; ++t)
      for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
          M[i * n + j] += op->lr_alpha[t] * op->lr_u[i * op->lr_rank + t] * op->lr_v[j * op->lr_rank + t];
    free(P);
    free(Pn);
  } else {
    const int64_t d = op->d, cols = d * (op->L + 1);
    double *B = (double *)calloc((size_t)(n * d), sizeof(double));
    double *Bn = (double *)calloc((size_t)(n * d), sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
      if (op->xdense) {
        for (int64_t f = 0; f < d; ++f) B[i * d + f] = op->xdense[i * d + f];
      } else {
        for (int64_t e = op->xrowptr[i]; e < op->xrowptr[i + 1]; ++e) B[i * d + op->xcolidx[e]] += op->xval[e];
      }
    }
    for (int l = 0; l <= op->L; ++l) {
      for (int64_t i = 0; i < n; ++i)
        for (int64_t f = 0; f < d; ++f) M[i * cols + l * d + f] = B[i * d + f];
      if (l < op->L) {
#pragma omp parallel for
        for (int64_t i = 0; i < n; ++i)
          for (int64_t f = 0; f < d; ++f) {
            double s = 0.0;
            for (int64_t t = 0; t < n; ++t) s += N[i * n + t] * B[t * d + f];
            Bn[i * d + f] = s;
          }
        double *t = B; B = Bn; Bn = t;
      }
    }
    free(B);
    free(Bn);
  }
  free(N);
  free(deg);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011) and Box-Muller       */
/* ------------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { /* key schedule: Weyl sequence bumps between rounds */
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Omega[i][j], rows x cols: counter (j/4, i_lo, i_hi, 0), key (seed_lo, seed_hi);
 * words (r0,r1) -> normals j%4 = 0,1 and (r2,r3) -> j%4 = 2,3 by Box-Muller:
 * u = (r + 1/2) 2^-32,  z_a = sqrt(-2 ln u_a) cos(2 pi u_b), z_b = ... sin(...). */
void orc_gaussian(uint64_t seed, int64_t rows, int64_t cols, double *out, int64_t ld) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  const double two_pi = 6.283185307179586476925286766559;
  for (int64_t i = 0; i < rows; ++i)
    for (int64_t q = 0; q < (cols + 3) / 4; ++q) {
      const uint32_t ctr[4] = {(uint32_t)q, (uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0u};
      uint32_t r[4];
      orc_philox4x32_10(ctr, key, r);
      double z[4];
      for (int h = 0; h < 2; ++h) {
        const double ua = ((double)r[2 * h] + 0.5) * 2.3283064365386962890625e-10;
        const double ub = ((double)r[2 * h + 1] + 0.5) * 2.3283064365386962890625e-10;
        const double rho = sqrt(-2.0 * log(ua));
        z[2 * h] = rho * cos(two_pi * ub);
        z[2 * h + 1] = rho * sin(two_pi * ub);
      }
      for (int t = 0; t < 4; ++t)
        if (4 * q + t < cols) out[i * ld + 4 * q + t] = z[t];
    }
}

/* ------------------------------------------------------------------------ */
/* Orthonormalisation (Alg. 2)                                               */
/* ------------------------------------------------------------------------ */

/* W = Q^T Q (c x c), Q is r x c row-major */
static void gram(const double *Q, int64_t r, int64_t c, double *W) {
#pragma omp parallel for
  for (int64_t a = 0; a < c; ++a)
    for (int64_t b = 0; b < c; ++b) {
      double s = 0.0;
      for (int64_t i = 0; i < r; ++i) s += Q[i * c + a] * Q[i * c + b];
      W[a * c + b] = s;
    }
}

/* Lower Cholesky W = L L^T; returns 0 on success, j+1 at a non-positive or
 * non-finite pivot j. */
int orc_cholesky(const double *W, int64_t c, double *Lf) {
  memset(Lf, 0, sizeof(double) * c * c);
  for (int64_t j = 0; j < c; ++j) {
    double s = W[j * c + j];
    for (int64_t t = 0; t < j; ++t) s -= Lf[j * c + t] * Lf[j * c + t];
    if (!(s > 0.0) || !isfinite(s)) return (int)(j + 1);
    const double ljj = sqrt(s);
    Lf[j * c + j] = ljj;
    for (int64_t i = j + 1; i < c; ++i) {
      double v = W[i * c + j];
      for (int64_t t = 0; t < j; ++t) v -= Lf[i * c + t] * Lf[j * c + t];
      Lf[i * c + j] = v / ljj;
    }
  }
  return 0;
}

/* Q <- Q (L^-1)^T: each row q^T becomes q^T L^-T, i.e. solve L y = q. */
static void apply_inv_lt(double *Q, int64_t r, int64_t c, const double *Lf) {
#pragma omp parallel for
  for (int64_t i = 0; i < r; ++i) {
    double *q = Q + i * c;
    for (int64_t j = 0; j < c; ++j) {
      double v = q[j];
      for (int64_t t = 0; t < j; ++t) v -= Lf[j * c + t] * q[t];
      q[j] = v / Lf[j * c + j];
    }
  }
}

/* One CholeskyQR pass (Alg. 2, right).  shift > 0 adds shift*I to the Gram.
 * On success, Rout (if non-NULL) receives R = L^T (upper, c x c).           */
int orc_cholqr(double *Q, int64_t r, int64_t c, double shift, double *Rout) {
  double *W = (double *)malloc(sizeof(double) * c * c);
  double *Lf = (double *)malloc(sizeof(double) * c * c);
  gram(Q, r, c, W);
  for (int64_t j = 0; j < c; ++j) W[j * c + j] += shift;
  const int info = orc_cholesky(W, c, Lf);
  if (info == 0) {
    apply_inv_lt(Q, r, c, Lf);
    if (Rout)
      for (int64_t a = 0; a < c; ++a)
        for (int64_t b = 0; b < c; ++b) Rout[a * c + b] = Lf[b * c + a];
  }
  free(W);
  free(Lf);
  return info;
}

/* R_acc <- R_new R_acc (both upper, c x c) */
static void rmul(const double *Rn, double *Racc, int64_t c) {
  double *T = (double *)malloc(sizeof(double) * c * c);
  for (int64_t a = 0; a < c; ++a)
    for (int64_t b = 0; b < c; ++b) {
      double s = 0.0;
      for (int64_t t = 0; t < c; ++t) s += Rn[a * c + t] * Racc[t * c + b];
      T[a * c + b] = s;
    }
  memcpy(Racc, T, sizeof(double) * c * c);
  free(T);
}

/* CholeskyQR2: two passes.  When the first Gram is not numerically positive
 * definite, a shifted pass (shift 11 (r c + c (c+1)) u ||Q||_F^2, u = 2^-53,
 * the shifted CholeskyQR of Fukaya et al. 2020) precedes two plain passes.
 * Returns the number of passes run (2 or 3), or -1 on failure.  Q = Qhat R. */
int orc_cholqr2(double *Q, int64_t r, int64_t c, double *R) {
  double *Rp = (double *)malloc(sizeof(double) * c * c);
  double *Racc = (double *)calloc((size_t)(c * c), sizeof(double));
  for (int64_t j = 0; j < c; ++j) Racc[j * c + j] = 1.0;
  int passes = 0;
  int info = orc_cholqr(Q, r, c, 0.0, Rp);
  if (info != 0) {
    double fro2 = 0.0;
    for (int64_t x = 0; x < r * c; ++x) fro2 += Q[x] * Q[x];
    const double shift = 11.0 * ((double)r * c + (double)c * (c + 1)) * 1.1102230246251565e-16 * fro2;
    info = orc_cholqr(Q, r, c, shift, Rp);
    if (info != 0) { free(Rp); free(Racc); return -1; }
    rmul(Rp, Racc, c);
    ++passes;
    info = orc_cholqr(Q, r, c, 0.0, Rp);
    if (info != 0) { free(Rp); free(Racc); return -1; }
  }
  rmul(Rp, Racc, c);
  ++passes;
  info = orc_cholqr(Q, r, c, 0.0, Rp);
  if (info != 0) { free(Rp); free(Racc); return -1; }
  rmul(Rp, Racc, c);
  ++passes;
  if (R) memcpy(R, Racc, sizeof(double) * c * c);
  free(Rp);
  free(Racc);
  return passes;
}

/* Householder QR of Q (r x c, r >= c): Q is overwritten by the thin
 * orthonormal factor, R (c x c upper) returned.  (Alg. 2, left.)            */
int orc_householder_qr(double *Q, int64_t r, int64_t c, double *R) {
  double *A = (double *)malloc(sizeof(double) * r * c);
  double *V = (double *)calloc((size_t)(r * c), sizeof(double)); /* reflectors */
  double *beta = (double *)calloc((size_t)c, sizeof(double));
  memcpy(A, Q, sizeof(double) * r * c);
  for (int64_t j = 0; j < c; ++j) {
    double nrm = 0.0;
    for (int64_t i = j; i < r; ++i) nrm += A[i * c + j] * A[i * c + j];
    nrm = sqrt(nrm);
    const double alpha = A[j * c + j] >= 0 ? -nrm : nrm;
    for (int64_t i = j; i < r; ++i) V[i * c + j] = A[i * c + j];
    V[j * c + j] -= alpha;
    double vv = 0.0;
    for (int64_t i = j; i < r; ++i) vv += V[i * c + j] * V[i * c + j];
    beta[j] = vv > 0 ? 2.0 / vv : 0.0;
    for (int64_t k = j; k < c; ++k) {
      double s = 0.0;
      for (int64_t i = j; i < r; ++i) s += V[i * c + j] * A[i * c + k];
      s *= beta[j];
      for (int64_t i = j; i < r; ++i) A[i * c + k] -= s * V[i * c + j];
    }
  }
  if (R)
    for (int64_t a = 0; a < c; ++a)
      for (int64_t b = 0; b < c; ++b) R[a * c + b] = b >= a ? A[a * c + b] : 0.0;
  /* thin Q = H_0 ... H_{c-1} [I; 0] */
  for (int64_t i = 0; i < r; ++i)
    for (int64_t k = 0; k < c; ++k) Q[i * c + k] = (i == k) ? 1.0 : 0.0;
  for (int64_t j = c - 1; j >= 0; --j)
    for (int64_t k = 0; k < c; ++k) {
      double s = 0.0;
      for (int64_t i = j; i < r; ++i) s += V[i * c + j] * Q[i * c + k];
      s *= beta[j];
      for (int64_t i = j; i < r; ++i) Q[i * c + k] -= s * V[i * c + j];
    }
  free(A);
  free(V);
  free(beta);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* One-sided Jacobi SVD (Hestenes), A is r x c with r >= c                   */
/* ------------------------------------------------------------------------ */

/* A = U diag(S) V^T.  U (r x c), S (c), V (c x c); singular values sorted
 * descending.  Cyclic sweeps over column pairs, rotation from Rutishauser's
 * formula, until every pair satisfies |g_p.g_q| <= tol ||g_p|| ||g_q||, with
 * tol floored at sqrt(r) eps (the rounding level of the dot product).  Pairs
 * of columns that are both below r eps ||A||_F carry only rounding noise and
 * are not rotated.  Returns the number of sweeps, or -1 when max_sweeps was
 * reached.                                                                  */
int orc_jacobi_svd(const double *A, int64_t r, int64_t c, double *U, double *S, double *V,
                   double tol, int max_sweeps) {
  double *G = (double *)malloc(sizeof(double) * r * c);
  double *J = (double *)calloc((size_t)(c * c), sizeof(double));
  memcpy(G, A, sizeof(double) * r * c);
  for (int64_t j = 0; j < c; ++j) J[j * c + j] = 1.0;
  double fro2 = 0.0;
  for (int64_t x = 0; x < r * c; ++x) fro2 += A[x] * A[x];
  const double eps = 2.220446049250313e-16;
  const double tiny = (double)r * eps * (double)r * eps * fro2;
  if (tol < sqrt((double)r) * eps) tol = sqrt((double)r) * eps;
  int sweep = 0, converged = 0;
  while (sweep < max_sweeps && !converged) {
    converged = 1;
    ++sweep;
    for (int64_t p = 0; p < c - 1; ++p)
      for (int64_t q = p + 1; q < c; ++q) {
        double alpha = 0.0, beta = 0.0, gamma = 0.0;
        for (int64_t i = 0; i < r; ++i) {
          const double gp = G[i * c + p], gq = G[i * c + q];
          alpha += gp * gp;
          beta += gq * gq;
          gamma += gp * gq;
        }
        if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha * beta)) continue;
        /* a column below the rounding level of A (norm^2 <= (r eps)^2 ||A||_F^2)
           is numerically zero: its direction is rounding noise, and rotating
           against it never converges and changes no singular value */
        if (alpha <= tiny || beta <= tiny) continue;
        converged = 0;
        const double zeta = (beta - alpha) / (2.0 * gamma);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        for (int64_t i = 0; i < r; ++i) {
          const double gp = G[i * c + p], gq = G[i * c + q];
          G[i * c + p] = cs * gp - sn * gq;
          G[i * c + q] = sn * gp + cs * gq;
        }
        for (int64_t i = 0; i < c; ++i) {
          const double jp = J[i * c + p], jq = J[i * c + q];
          J[i * c + p] = cs * jp - sn * jq;
          J[i * c + q] = sn * jp + cs * jq;
        }
      }
  }
  /* column norms, sort descending */
  double *nrm = (double *)malloc(sizeof(double) * c);
  int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * c);
  for (int64_t j = 0; j < c; ++j) {
    double s = 0.0;
    for (int64_t i = 0; i < r; ++i) s += G[i * c + j] * G[i * c + j];
    nrm[j] = sqrt(s);
    ord[j] = j;
  }
  for (int64_t a = 1; a < c; ++a) { /* insertion sort, stable */
    const int64_t x = ord[a];
    int64_t b = a - 1;
    while (b >= 0 && nrm[ord[b]] < nrm[x]) { ord[b + 1] = ord[b]; --b; }
    ord[b + 1] = x;
  }
  for (int64_t k = 0; k < c; ++k) {
    const int64_t j = ord[k];
    S[k] = nrm[j];
    for (int64_t i = 0; i < r; ++i) U[i * c + k] = nrm[j] > 0 ? G[i * c + j] / nrm[j] : 0.0;
    for (int64_t i = 0; i < c; ++i) V[i * c + k] = J[i * c + j];
  }
  free(nrm);
  free(ord);
  free(G);
  free(J);
  return converged ? sweep : -1;
}

/* ------------------------------------------------------------------------ */
/* iSVD (Alg. 1) with block width l = k + p                                  */
/* ------------------------------------------------------------------------ */

/* U (r x k), S (k), V (c x k), all row-major with ld = k.  Returns 0, or a
 * negative code when an orthonormalisation or the small SVD failed.
 * info[0] = number of CholeskyQR passes run in total.                      */
int orc_isvd(const orc_op *op, int32_t k, int32_t p, int32_t iters, uint64_t seed,
             double *U, double *S, double *V, int32_t *info) {
  const int64_t r = orc_rows(op), c = orc_cols(op), l = k + p;
  double *Q = (double *)malloc(sizeof(double) * c * l);
  double *Y = (double *)malloc(sizeof(double) * (r > c ? r : c) * l);
  int passes = 0, rc;
  orc_gaussian(seed, c, l, Q, l); /* Q ~ N(0,1)^{c x l} */
  for (int32_t it = 0; it < iters; ++it) {
    orc_apply(op, Q, l, Y, 0); /* r x l */
    if ((rc = orc_cholqr2(Y, r, l, NULL)) < 0) goto fail;
    passes += rc;
    orc_apply(op, Y, l, Q, 1); /* c x l */
    if ((rc = orc_cholqr2(Q, c, l, NULL)) < 0) goto fail;
    passes += rc;
  }
  orc_apply(op, Q, l, Y, 0);
  if ((rc = orc_cholqr2(Y, r, l, NULL)) < 0) goto fail;
  passes += rc;
  {
    /* B = (M^T Q)^T (l x c); SVD(B) = UB diag(s) VB^T through one-sided Jacobi
     * of B^T (c x l): B^T = VB diag(s) UB^T. */
    double *Bt = (double *)malloc(sizeof(double) * c * l);
    double *Wv = (double *)malloc(sizeof(double) * c * l);
    double *s = (double *)malloc(sizeof(double) * l);
    double *UB = (double *)malloc(sizeof(double) * l * l);
    orc_apply(op, Y, l, Bt, 1);
    const int sw = orc_jacobi_svd(Bt, c, l, Wv, s, UB, 1e-15, 100);
    if (sw < 0) { free(Bt); free(Wv); free(s); free(UB); rc = -2; goto fail; }
    /* U = Q UB (r x l), keep the first k columns */
    for (int64_t i = 0; i < r; ++i)
      for (int64_t j = 0; j < k; ++j) {
        double acc = 0.0;
        for (int64_t t = 0; t < l; ++t) acc += Y[i * l + t] * UB[t * l + j];
        U[i * k + j] = acc;
      }
    for (int64_t j = 0; j < k; ++j) S[j] = s[j];
    for (int64_t i = 0; i < c; ++i)
      for (int64_t j = 0; j < k; ++j) V[i * k + j] = Wv[i * l + j];
    free(Bt); free(Wv); free(s); free(UB);
  }
  if (info) info[0] = passes;
  free(Q);
  free(Y);
  return 0;
fail:
  free(Q);
  free(Y);
  return rc < 0 ? rc : -1;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
