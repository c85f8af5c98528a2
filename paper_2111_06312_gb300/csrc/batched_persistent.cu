// Many independent rank-k SVDs (Alg. 1 on each problem) in ONE persistent
// kernel: the batched form with per-problem stage counters and bounded waits.
//
// A problem is taken by a team of T CTAs (one per 16,384 rows, 1..32), member m
// owning rows [n m / T, n (m + 1) / T) of every block.  The CTAs of the grid
// (all resident: cooperative launch, one per SM) pull (problem, member) items
// from one queue in which a team's members are consecutive and the largest
// problems come first, and run the whole of Alg. 1 for their member:
//   start block (Philox4x32-10 + Box-Muller, as isvd_gaussian),
//   M Q / M^T Q by Horner (Eq. 3; T = D^-1 A or A-hat) with the all-ones term,
//   CholeskyQR2 with the shift of Alg. 2 (the same gates as isvd_svd),
//   Rayleigh-Ritz: QR of B^T, one-sided Jacobi of R, U = Q Vo, V = Qt Uo.
// Wherever a step reads rows that other members wrote (a sparse product
// gathers any row; the Gram and the column sums are summed over members) the
// team meets at its stage counter: every member adds one and waits, with a
// bounded spin, until all T have.  A wait that runs out marks the problem
// abandoned (its status ISVD_ERR_TIMEOUT); its members drop it and take the
// next item, so the kernel always ends.  The queue cannot deadlock: items are
// handed out in order and a team's members are consecutive, so every team
// whose members have all been taken runs to the end, and an idle CTA always
// takes the next item.
//
// Arithmetic: SIMT FP32 products with FP64 accumulation where the
// tensor-core path accumulates in FP64 (Gram partials promoted every 512
// rows, column sums), FP64 Cholesky, inverse and Jacobi in shared memory.
// The results equal isvd_svd's up to rounding (the order of the sums differs).
#include <algorithm>
#include <vector>

#include "internal.h"
#include "jacobi_common.cuh"
#include "philox.cuh"

namespace isvd {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxL = ISVD_PERSISTENT_MAX_BLOCK;
constexpr int kMaxTeam = 32;
constexpr int kDefaultTeamRows = 16384;  // rows per team member (measured best of 1,024..16,384)
constexpr int kStageRows = 128;         // rows of a block staged in shared memory
constexpr int kPromoteChunks = 4;       // Gram: FP32 sums promoted to FP64 every 512 rows
constexpr uint32_t kDefaultSpin = 1u << 22;

struct Problem {
  int32_t n, l, ld, k, team, norm, degree, iters;
  float coeff[ISVD_MAX_DEGREE];  // c_1 .. c_K
  float ones;                    // alpha of alpha 1 1^T (0: none)
  uint64_t seed;
  const int32_t *rowptr, *colidx;
  const float *inv_d, *s;  // 1/deg, (deg + 1)^-1/2
  float *U, *S, *V;        // outputs: n x k, k, n x k (dense)
  float *Qr, *Qc, *Z1, *Z2;  // n x ld blocks
  double *part;            // [2][team][l][l] Gram partials, by pass parity
  double *csum;            // [team][l] column-sum partials
  double *Racc[2];         // l x l, ping-pong
  float *Lk, *Rk;          // l x k
  isvd_info *info;
  unsigned *arrive;        // the team's stage counter
  int *err;                // the problem was abandoned
};

struct Item {
  int32_t problem, member;
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Shared memory of a CTA (dynamic): W (l x l FP64), R^-1 / B (l x l FP32), a
// staged block of kStageRows rows (FP32, also FP64 scratch), small vectors.
struct Smem {
  double *W;     // Gram sum, Cholesky factor, Jacobi columns
  float *B;      // R^-1 (upper) or the closing product's small matrix
  float *stage;  // kStageRows x ld (row-major) or ld x (kStageRows + 4) (transposed)
  double *vec;   // 2 l + 32 doubles: column sums, norms, a reduction
  float *ones;   // l floats: alpha (1^T G)
};

__host__ __device__ inline size_t stage_floats(int ld) {
  return (size_t)ld * (kStageRows + 4) > (size_t)kStageRows * ld ? (size_t)ld * (kStageRows + 4)
                                                                 : (size_t)kStageRows * ld;
}
// every part starts on a 16-byte boundary (float4 accesses): double counts even
__host__ __device__ inline size_t w_doubles(int l) { return ((size_t)l * l + 1) & ~(size_t)1; }
__host__ __device__ inline size_t vec_doubles(int l) { return 2 * (size_t)l + 32; }
__host__ __device__ inline size_t smem_bytes(int l, int ld) {
  return sizeof(double) * (w_doubles(l) + vec_doubles(l)) + sizeof(float) * (size_t)l * ld +
         sizeof(float) * stage_floats(ld) + sizeof(float) * ld + 64;
}

struct Ctx {
  const Problem &P;
  int member;
  unsigned phase;     // team meetings so far
  uint32_t spin;
  int phantom;        // test only: wait for one member more than the team has
  int64_t r0, r1;     // this member's rows
  Smem sm;
};

// The team meets: every member adds one to the counter and waits until all
// have (bounded).  false: the problem was abandoned (by this or another member).
__device__ bool team_meet(Ctx &c) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const int T = c.P.team + c.phantom;
    if (T > 1) {
      __threadfence();
      atomicAdd(c.P.arrive, 1u);
      ++c.phase;
      const unsigned target = c.phase * (unsigned)T;
      uint32_t spins = 0;
      while (ld_acquire_u32(c.P.arrive) < target) {
        if (*(volatile int *)c.P.err || ++spins > c.spin) {
          atomicExch(c.P.err, 1);
          atomicExch(&c.P.info->status, (int)ISVD_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    } else {
      ++c.phase;
    }
    if (ok && *(volatile int *)c.P.err) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

// ---- start block: Qc rows of this member ~ N(0,1), padding columns zero ----
__device__ void start_block(Ctx &c) {
  const Problem &P = c.P;
  const uint32_t k0 = (uint32_t)P.seed, k1 = (uint32_t)(P.seed >> 32);
  const int nq = P.ld / 4;
  const int64_t total = (c.r1 - c.r0) * nq;
  for (int64_t idx = threadIdx.x; idx < total; idx += kThreads) {
    const int64_t i = c.r0 + idx / nq;
    const int q = (int)(idx % nq);
    float z[4] = {0.f, 0.f, 0.f, 0.f};
    if (4 * q < P.l) gaussian_quad(k0, k1, i, q, z);
    float4 v;
    v.x = 4 * q + 0 < P.l ? z[0] : 0.f;
    v.y = 4 * q + 1 < P.l ? z[1] : 0.f;
    v.z = 4 * q + 2 < P.l ? z[2] : 0.f;
    v.w = 4 * q + 3 < P.l ? z[3] : 0.f;
    *reinterpret_cast<float4 *>(P.Qc + i * P.ld + 4 * q) = v;
  }
}

// ---- column sums of G (the all-ones term): member partials, then the sum ----
// Thread (column b, row group g) adds 32-row FP32 pieces into an FP64 sum.
__device__ bool column_sums(Ctx &c, const float *G) {
  const Problem &P = c.P;
  const int l = P.l;
  const int groups = kThreads / l;
  const int b = threadIdx.x % l, g = threadIdx.x / l;
  double *acc = c.sm.vec;  // [groups] reduced one group at a time below
  double mine = 0.0;
  __syncthreads();  // the rows of G that this CTA has just written are complete
  if (g < groups) {
    for (int64_t i0 = c.r0 + (int64_t)g * 32; i0 < c.r1; i0 += (int64_t)groups * 32) {
      float piece = 0.f;
      const int64_t i1 = min(c.r1, i0 + 32);
      for (int64_t i = i0; i < i1; ++i) piece += __ldcg(G + i * P.ld + b);
      mine += (double)piece;
    }
  }
  for (int t = threadIdx.x; t < l; t += kThreads) acc[t] = 0.0;
  __syncthreads();
  for (int gg = 0; gg < groups; ++gg) {  // fixed order over groups
    if (g == gg) acc[b] += mine;
    __syncthreads();
  }
  double *mypart = P.csum + (size_t)c.member * l;
  for (int t = threadIdx.x; t < l; t += kThreads) mypart[t] = acc[t];
  if (!team_meet(c)) return false;
  for (int t = threadIdx.x; t < l; t += kThreads) {
    double s = 0.0;
    for (int m = 0; m < P.team; ++m) s += __ldcg(P.csum + (size_t)m * l + t);
    c.sm.ones[t] = (float)(P.ones * s);
  }
  __syncthreads();
  return true;
}

// ---- one sparse product of the Horner chain, rows of this member ----
// out_i = mult (op src)_i + axc G_i [+ ones_b], op = T (norm row), T^T, or A-hat.
// A group of Gl lanes (one 16-byte column chunk each) takes two rows at a
// time, A and B, so that their index and gather round trips overlap: the
// group loads Gl column indices of each row at once (one per lane), then
// every lane gathers its chunk of four rows of A and four of B at a time.
__device__ __forceinline__ float4 fma4(float w, float4 v, float4 a) {
  return make_float4(fmaf(w, v.x, a.x), fmaf(w, v.y, a.y), fmaf(w, v.z, a.z), fmaf(w, v.w, a.w));
}

__device__ void sparse_epilogue(Ctx &c, const float *src, float *out, float mult, const float *G, float axc,
                                bool transpose, bool add_ones, int64_t i, int gl, float4 acc, float4 g) {
  const Problem &P = c.P;
  float sc;
  if (P.norm == ISVD_NORM_ROW) {
    sc = transpose ? 1.f : __ldg(P.inv_d + i);
  } else {
    const float si = __ldg(P.s + i);
    if (P.norm == ISVD_NORM_SYM_SELFLOOP)
      acc = fma4(si, __ldcg(reinterpret_cast<const float4 *>(src + i * P.ld) + gl), acc);
    sc = si;
  }
  sc *= mult;
  float4 r = make_float4(sc * acc.x, sc * acc.y, sc * acc.z, sc * acc.w);
  if (G) r = fma4(axc, g, r);
  if (add_ones) {
    const int b = 4 * gl;
    if (b + 0 < P.l) r.x += c.sm.ones[b + 0];
    if (b + 1 < P.l) r.y += c.sm.ones[b + 1];
    if (b + 2 < P.l) r.z += c.sm.ones[b + 2];
    if (b + 3 < P.l) r.w += c.sm.ones[b + 3];
  }
  reinterpret_cast<float4 *>(out + i * P.ld)[gl] = r;
}

__device__ void sparse_step(Ctx &c, const float *src, float *out, float mult, const float *G, float axc,
                            bool transpose, bool add_ones) {
  const Problem &P = c.P;
  const int nq = P.ld / 4;
  int Gl = 8;
  while (Gl < nq) Gl <<= 1;  // lanes per row: 8, 16 or 32
  const int rpw = 32 / Gl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int sub = lane / Gl, gl = lane - sub * Gl;
  const int lead = sub * Gl;
  const bool active = gl < nq;
  const bool row = P.norm == ISVD_NORM_ROW;
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  auto weight = [&](int j) { return row ? (transpose ? __ldg(P.inv_d + j) : 1.f) : __ldg(P.s + j); };
  for (int64_t base = c.r0 + (int64_t)warp * 2 * rpw; base < c.r1; base += (int64_t)kWarps * 2 * rpw) {
    const int64_t iA = base + sub, iB = base + rpw + sub;
    const bool hA = iA < c.r1, hB = iB < c.r1;
    int eA = 0, lenA = 0, eB = 0, lenB = 0;
    if (hA) {
      eA = __ldg(P.rowptr + iA);
      lenA = __ldg(P.rowptr + iA + 1) - eA;
    }
    if (hB) {
      eB = __ldg(P.rowptr + iB);
      lenB = __ldg(P.rowptr + iB + 1) - eB;
    }
    float4 gA = zero, gB = zero;  // the axpy operand, loaded ahead of the gathers
    if (G && active) {
      if (hA) gA = __ldcg(reinterpret_cast<const float4 *>(G + iA * P.ld) + gl);
      if (hB) gB = __ldcg(reinterpret_cast<const float4 *>(G + iB * P.ld) + gl);
    }
    float4 accA = zero, accB = zero;
    const int len = max(lenA, lenB);
    for (int off = 0; __any_sync(0xffffffffu, off < len); off += Gl) {
      int jA = -1, jB = -1;
      float wA = 0.f, wB = 0.f;
      if (off + gl < lenA) jA = __ldg(P.colidx + eA + off + gl);
      if (off + gl < lenB) jB = __ldg(P.colidx + eB + off + gl);
      if (jA >= 0) wA = weight(jA);
      if (jB >= 0) wB = weight(jB);
      const int cA = max(0, min(Gl, lenA - off)), cB = max(0, min(Gl, lenB - off));
      const int wcnt = __reduce_max_sync(0xffffffffu, max(cA, cB));  // the warp steps to its longest row
      for (int u0 = 0; u0 < wcnt; u0 += 4) {
        int ja[4], jb[4];
        float wa[4], wb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int sl = lead + ((u0 + u) & (Gl - 1));
          ja[u] = __shfl_sync(0xffffffffu, jA, sl);
          wa[u] = __shfl_sync(0xffffffffu, wA, sl);
          jb[u] = __shfl_sync(0xffffffffu, jB, sl);
          wb[u] = __shfl_sync(0xffffffffu, wB, sl);
          if (u0 + u >= cA) ja[u] = -1;
          if (u0 + u >= cB) jb[u] = -1;
        }
        if (active) {
          float4 va[4], vb[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            va[u] = ja[u] >= 0 ? __ldcg(reinterpret_cast<const float4 *>(src + (int64_t)ja[u] * P.ld) + gl) : zero;
            vb[u] = jb[u] >= 0 ? __ldcg(reinterpret_cast<const float4 *>(src + (int64_t)jb[u] * P.ld) + gl) : zero;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            accA = fma4(wa[u], va[u], accA);
            accB = fma4(wb[u], vb[u], accB);
          }
        }
      }
    }
    if (!active) continue;
    if (hA) sparse_epilogue(c, src, out, mult, G, axc, transpose, add_ones, iA, gl, accA, gA);
    if (hB) sparse_epilogue(c, src, out, mult, G, axc, transpose, add_ones, iB, gl, accB, gB);
  }
}

// out = M G (or M^T G) by Horner: Z = c_K op G + c_{K-1} G; Z = op Z + c_{k-1} G;
// out = op Z [+ alpha 1 1^T G].  Every step gathers rows of every member.
__device__ bool apply(Ctx &c, const float *G, float *out, bool transpose) {
  const Problem &P = c.P;
  const int K = P.degree;
  const bool ones = P.ones != 0.f;
  if (ones) {
    if (!column_sums(c, G)) return false;  // ends with a meeting: G is complete
  } else if (!team_meet(c)) {
    return false;
  }
  if (K == 1) {
    sparse_step(c, G, out, P.coeff[0], nullptr, 0.f, transpose, ones);
    return true;
  }
  float *zb[2] = {P.Z1, P.Z2};
  const float *cur = G;
  int which = 0;
  for (int step = K; step >= 1; --step) {
    const bool first = step == K, last = step == 1;
    float *dst = last ? out : zb[which];
    sparse_step(c, cur, dst, first ? P.coeff[K - 1] : 1.f, last ? nullptr : G, last ? 0.f : P.coeff[step - 2],
                transpose, last && ones);
    if (!last && !team_meet(c)) return false;
    cur = dst;
    which ^= 1;
  }
  return true;
}

// ---- Gram partial of this member's rows: W_m = Q_m^T Q_m (FP64, upper) ----
// 4 x 4 tiles of the upper triangle, `groups` copies over interleaved rows;
// FP32 sums promoted to FP64 every kPromoteChunks staged chunks.
__device__ void gram_partial(Ctx &c, const float *Q, double *out) {
  const Problem &P = c.P;
  const int l = P.l, ld = P.ld;
  const int nb4 = (l + 3) / 4;
  const int ntile = nb4 * (nb4 + 1) / 2;
  const int groups = max(1, kThreads / ntile);
  const int t = threadIdx.x % ntile, grp = threadIdx.x / ntile;
  const bool on = grp < groups && (int)threadIdx.x < ntile * groups;
  // tile t -> (bi, bj), bi <= bj
  int bi = 0, rem = t;
  while (rem >= nb4 - bi) {
    rem -= nb4 - bi;
    ++bi;
  }
  const int bj = bi + rem;
  float a32[4][4];
  double a64[4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      a32[x][y] = 0.f;
      a64[x][y] = 0.0;
    }
  int chunk = 0;
  for (int64_t s0 = c.r0; s0 < c.r1; s0 += kStageRows, ++chunk) {
    const int rows = (int)(c.r1 - s0 < kStageRows ? c.r1 - s0 : kStageRows);
    __syncthreads();
    for (int idx = threadIdx.x; idx < rows * (ld / 4); idx += kThreads) {
      const int rr = idx / (ld / 4), q = idx - rr * (ld / 4);
      reinterpret_cast<float4 *>(c.sm.stage + (size_t)rr * ld)[q] =
          __ldcg(reinterpret_cast<const float4 *>(Q + (s0 + rr) * ld) + q);
    }
    __syncthreads();
    if (on) {
      for (int rr = grp; rr < rows; rr += groups) {
        const float4 x = reinterpret_cast<const float4 *>(c.sm.stage + (size_t)rr * ld)[bi];
        const float4 y = reinterpret_cast<const float4 *>(c.sm.stage + (size_t)rr * ld)[bj];
        const float xa[4] = {x.x, x.y, x.z, x.w}, ya[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) a32[p][q] = fmaf(xa[p], ya[q], a32[p][q]);
      }
    }
    if ((chunk + 1) % kPromoteChunks == 0 || s0 + kStageRows >= c.r1) {
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          a64[p][q] += (double)a32[p][q];
          a32[p][q] = 0.f;
        }
    }
  }
  // groups summed into W in a fixed order, then written out
  for (int idx = threadIdx.x; idx < l * l; idx += kThreads) c.sm.W[idx] = 0.0;
  __syncthreads();
  for (int g = 0; g < groups; ++g) {
    if (on && grp == g)
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int a = 4 * bi + p, b = 4 * bj + q;
          if (a < l && b < l && a <= b) c.sm.W[a * l + b] += a64[p][q];
        }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < l * l; idx += kThreads) out[idx] = c.sm.W[idx];
}

// ---- the l x l FP64 step of one CholeskyQR pass (every member alike) ----
// W = sum of the members' partials (+ shift), Cholesky in place (upper R),
// R^-1 into B (FP32), and when `racc`, Racc <- R Racc (member 0).
// Returns false when the problem was abandoned; sets *shifted, *reorth.
struct PassState {
  int last_flag;  // last pass that needed a shift or a re-orthogonalisation
  int racc_cur;   // which Racc buffer holds the product
};

__device__ bool chol_step(Ctx &c, const double *parts, int pass, bool racc, PassState &ps) {
  const Problem &P = c.P;
  const int l = P.l;
  double *W = c.sm.W;
  double *x = reinterpret_cast<double *>(c.sm.stage);  // scratch: [kWarps][l] back substitution, then invd
  __shared__ int s_fail;
  __shared__ double s_trace;
  double shift = 0.0;
  bool ok = false;
  for (int attempt = 0; attempt < 10 && !ok; ++attempt) {
    for (int idx = threadIdx.x; idx < l * l; idx += kThreads) {
      const int a = idx / l, b = idx - a * l;
      double s = 0.0;
      const int u = a <= b ? a * l + b : b * l + a;  // partials hold the upper triangle
      for (int m = 0; m < P.team; ++m) s += __ldcg(parts + (size_t)m * l * l + u);
      W[idx] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double tr = 0.0;
      for (int j = 0; j < l; ++j) tr += W[j * l + j];
      s_trace = tr;
      s_fail = 0;
    }
    __syncthreads();
    if (attempt == 1) shift = 16.0 * l * 5.9604644775390625e-08 * fabs(s_trace);
    if (attempt > 1) shift *= 10.0;
    if (shift > 0.0)
      for (int j = threadIdx.x; j < l; j += kThreads) W[j * l + j] += shift;
    __syncthreads();
    for (int j = 0; j < l; ++j) {
      const double d = W[j * l + j];
      if (!(d > 0.0) || !isfinite(d)) {
        if (threadIdx.x == 0) s_fail = 1;
        __syncthreads();
        break;
      }
      const double inv = rsqrt(d);
      __syncthreads();  // every thread has read d
      for (int col = j + 1 + (int)threadIdx.x; col < l; col += kThreads) W[j * l + col] *= inv;
      if (threadIdx.x == 0) W[j * l + j] = d * inv;
      __syncthreads();
      const int m = l - j - 1;
      for (int idx = threadIdx.x; idx < m * m; idx += kThreads) {
        const int ii = idx / m, cc = idx - ii * m;
        if (cc >= ii) {
          const int i = j + 1 + ii, col = j + 1 + cc;
          W[i * l + col] -= W[j * l + i] * W[j * l + col];
        }
      }
      __syncthreads();
    }
    ok = s_fail == 0;
    __syncthreads();
  }
  if (!ok)  // no shift cured it: R = I, the status says so
    for (int idx = threadIdx.x; idx < l * l; idx += kThreads) W[idx] = (idx / l == idx % l) ? 1.0 : 0.0;
  // strictly lower part to zero (the sums above wrote it)
  for (int idx = threadIdx.x; idx < l * l; idx += kThreads)
    if (idx / l > idx % l) W[idx] = 0.0;
  __syncthreads();
  bool reorth = false;
  if (ok && pass >= 2) {
    __shared__ int s_far;
    if (threadIdx.x == 0) s_far = 0;
    __syncthreads();
    for (int idx = threadIdx.x; idx < l * l; idx += kThreads)
      if (fabs(W[idx] - ((idx / l == idx % l) ? 1.0 : 0.0)) > 0.25) s_far = 1;
    __syncthreads();
    reorth = s_far != 0;
  }
  if (c.member == 0 && threadIdx.x == 0) {
    if (!ok) {
      atomicExch(&P.info->status, (int)ISVD_ERR_NOT_POSITIVE_DEFINITE);
    } else {
      if (shift > 0.0) atomicAdd(&P.info->chol_shifts, 1);
      atomicAdd(&P.info->cholqr_passes, 1);
    }
  }
  if (ok && shift > 0.0) ps.last_flag = max(ps.last_flag, pass);
  if (reorth) ps.last_flag = max(ps.last_flag, pass - 1);
  // R^-1: one warp per column, right-looking (lanes over the rows of the running sums)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *invd = x + (size_t)kWarps * l;
  for (int i = threadIdx.x; i < l; i += kThreads) invd[i] = 1.0 / W[i * l + i];
  __syncthreads();
  double *xv = x + (size_t)warp * l;
  for (int col = warp; col < l; col += kWarps) {
    for (int i = lane; i < col; i += 32) xv[i] = 0.0;
    __syncwarp();
    for (int t = col; t >= 0; --t) {
      const double xt = t == col ? invd[col] : -xv[t] * invd[t];
      for (int i = lane; i < t; i += 32) xv[i] = fma(W[i * l + t], xt, xv[i]);
      __syncwarp();
      if (lane == 0) xv[t] = xt;
      __syncwarp();
    }
    for (int i = lane; i < l; i += 32) c.sm.B[i * P.ld + col] = i <= col ? (float)xv[i] : 0.f;
    __syncwarp();
  }
  for (int idx = threadIdx.x; idx < l * (P.ld - l); idx += kThreads) {
    const int i = idx / (P.ld - l), col = l + idx % (P.ld - l);
    c.sm.B[i * P.ld + col] = 0.f;
  }
  // Racc <- R Racc (member 0 keeps the product)
  if (racc && c.member == 0) {
    const double *Ro = P.Racc[ps.racc_cur];
    double *Rn = P.Racc[ps.racc_cur ^ 1];
    for (int idx = threadIdx.x; idx < l * l; idx += kThreads) {
      const int i = idx / l, col = idx - i * l;
      double s = 0.0;
      for (int t = i; t <= col; ++t) s += W[i * l + t] * Ro[(size_t)t * l + col];
      Rn[idx] = i <= col ? s : 0.0;
    }
    ps.racc_cur ^= 1;
  }
  __syncthreads();
  return true;
}

// ---- rows of this member: out = Q B (B l x w in shared memory, ld ldb) ----
// Staged transposed (column-major, kStageRows + 4 pitch); a thread takes 4
// rows x 4 columns.  `upper`: B upper triangular (the sum stops at the column).
__device__ void rows_times_small(Ctx &c, const float *Q, const float *B, int ldb, int w, bool upper, float *out,
                                 int ldo) {
  const Problem &P = c.P;
  const int l = P.l, ld = P.ld;
  const int pitch = kStageRows + 4;
  const int nq = (w + 3) / 4;
  for (int64_t s0 = c.r0; s0 < c.r1; s0 += kStageRows) {
    const int rows = (int)(c.r1 - s0 < kStageRows ? c.r1 - s0 : kStageRows);
    __syncthreads();
    for (int idx = threadIdx.x; idx < rows * ld; idx += kThreads) {
      const int rr = idx / ld, col = idx - rr * ld;
      c.sm.stage[(size_t)col * pitch + rr] = __ldcg(Q + (s0 + rr) * ld + col);
    }
    for (int idx = threadIdx.x; idx < (kStageRows - rows) * ld; idx += kThreads) {
      const int rr = rows + idx / ld, col = idx % ld;
      c.sm.stage[(size_t)col * pitch + rr] = 0.f;
    }
    __syncthreads();
    const int items = (kStageRows / 4) * nq;
    for (int it = threadIdx.x; it < items; it += kThreads) {
      const int rq = it % (kStageRows / 4), cq = it / (kStageRows / 4);
      if (4 * rq >= rows) continue;
      float acc[4][4];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
      const int tmax = upper ? min(l, 4 * cq + 4) : l;
      for (int t = 0; t < tmax; ++t) {
        const float4 a = *reinterpret_cast<const float4 *>(c.sm.stage + (size_t)t * pitch + 4 * rq);
        const float4 b = *reinterpret_cast<const float4 *>(B + (size_t)t * ldb + 4 * cq);
        const float aa[4] = {a.x, a.y, a.z, a.w}, bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(aa[p], bb[q], acc[p][q]);
      }
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int rr = 4 * rq + p;
        if (rr >= rows) break;
        float *o = out + (s0 + rr) * ldo + 4 * cq;
        if (4 * cq + 4 <= w && (ldo & 3) == 0 && ((uintptr_t)o & 15) == 0) {
          *reinterpret_cast<float4 *>(o) = make_float4(acc[p][0], acc[p][1], acc[p][2], acc[p][3]);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (4 * cq + q < w) o[q] = acc[p][q];
        }
      }
    }
  }
}

// ---- CholeskyQR2 with the gates of isvd_svd (passes 3, 4 after a shift or a
// factor far from I); `racc`: R accumulated into Racc (member 0) ----
__device__ bool orthonormalize(Ctx &c, float *Q, bool racc, PassState &ps) {
  const Problem &P = c.P;
  const int l = P.l;
  ps.last_flag = 0;
  if (racc && c.member == 0) {
    double *R0 = P.Racc[ps.racc_cur];
    for (int idx = threadIdx.x; idx < l * l; idx += kThreads) R0[idx] = (idx / l == idx % l) ? 1.0 : 0.0;
  }
  for (int pass = 1; pass <= 4; ++pass) {
    if (pass > 2 && ps.last_flag + 2 < pass) break;  // the same decision in every member
    double *parts = P.part + (size_t)(pass & 1) * P.team * l * l;
    gram_partial(c, Q, parts + (size_t)c.member * l * l);
    if (!team_meet(c)) return false;
    if (!chol_step(c, parts, pass, racc, ps)) return false;
    __syncthreads();
    rows_times_small(c, Q, c.sm.B, P.ld, P.ld, true, Q, P.ld);
  }
  return true;
}

// ---- Rayleigh-Ritz: SVD of R (= Racc) by one-sided Jacobi on the columns of
// R^T, one CTA (member 0): Lk = Vo[:, :k], Rk = Uo[:, :k], S ----
__device__ void rayleigh_ritz(Ctx &c, const double *R) {
  const Problem &P = c.P;
  const int l = P.l, k = P.k;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double *Gs = c.sm.W;              // column p of G = row p of R
  double *nrm = c.sm.vec;           // l squared norms
  double *red = c.sm.vec + l;       // scratch
  for (int idx = threadIdx.x; idx < l * l; idx += kThreads) Gs[idx] = R[idx];
  __syncthreads();
  const double fro2 = frobenius2(R, l, red);
  const double eps = 2.220446049250313e-16;
  const double tol = fmax(1e-15, sqrt((double)l) * eps);
  const double tiny = (double)l * eps * (double)l * eps * fro2;
  const int players = (l + 1) & ~1;
  __shared__ int s_any;
  for (int sweep = 0; sweep < 60; ++sweep) {
    for (int p = warp; p < l; p += kWarps) {
      double s2 = 0.0;
      for (int i = lane; i < l; i += 32) s2 += Gs[p * l + i] * Gs[p * l + i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) nrm[p] = s2;
    }
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    int rotated = 0;
    for (int r = 0; r < players - 1; ++r) {
      for (int pr = warp; pr < players / 2; pr += kWarps) {
        int p, q;
        tourney(r, pr, players, p, q);
        if (p >= l || q >= l) continue;
        double *gp = Gs + p * l, *gq = Gs + q * l;
        double ga = 0.0;
        for (int i = lane; i < l; i += 32) ga += gp[i] * gq[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
        double t, cs, sn;
        if (!jacobi_angle(ga, nrm[p], nrm[q], tol, tiny, t, cs, sn)) continue;
        rotated = 1;
        for (int i = lane; i < l; i += 32) {
          const double a = gp[i], b = gq[i];
          gp[i] = cs * a - sn * b;
          gq[i] = sn * a + cs * b;
        }
        __syncwarp();
        if (lane == 0) {
          const double al = nrm[p], be = nrm[q];
          nrm[p] = al - t * ga;
          nrm[q] = be + t * ga;
        }
        __syncwarp();
      }
      __syncthreads();
    }
    if (rotated) s_any = 1;
    __syncthreads();
    if (!s_any) break;
    __syncthreads();
  }
  // norms, order (descending, stable), outputs
  for (int p = warp; p < l; p += kWarps) {
    double s2 = 0.0;
    for (int i = lane; i < l; i += 32) s2 += Gs[p * l + i] * Gs[p * l + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane == 0) nrm[p] = sqrt(s2);
  }
  __syncthreads();
  __shared__ int perm[kMaxL];
  for (int p = threadIdx.x; p < l; p += kThreads) {
    const double xp = nrm[p] == nrm[p] ? nrm[p] : -1.0;
    int rank = 0;
    for (int q = 0; q < l; ++q) {
      const double xq = nrm[q] == nrm[q] ? nrm[q] : -1.0;
      rank += (xq > xp || (xq == xp && q < p)) ? 1 : 0;
    }
    perm[rank] = p;
  }
  __syncthreads();
  // column kk < k: Vo = w_p / sigma, Uo = R w_p / sigma^2 (one warp per entry row)
  for (int kk = 0; kk < k; ++kk) {
    const int p = perm[kk];
    const double sg = nrm[p];
    const double *w = Gs + p * l;
    for (int i = warp; i < l; i += kWarps) {
      double u = 0.0;
      for (int t = lane; t < l; t += 32) u += R[(size_t)i * l + t] * w[t];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
      if (lane == 0) {
        P.Lk[(size_t)i * k + kk] = (float)(sg > 0.0 ? w[i] / sg : 0.0);
        P.Rk[(size_t)i * k + kk] = (float)(sg > 0.0 ? u / (sg * sg) : 0.0);
      }
    }
    if (threadIdx.x == 0) P.S[kk] = (float)sg;
  }
  if (threadIdx.x == 0) P.info->iters_done = P.iters;
}

__device__ void run_member(const Problem &P, int member, uint32_t spin, int phantom, Smem sm) {
  Ctx c{P, member, 0u, spin, phantom, (int64_t)P.n * member / P.team, (int64_t)P.n * (member + 1) / P.team, sm};
  PassState ps{0, 0};
  start_block(c);
  for (int it = 0; it < P.iters; ++it) {
    if (!apply(c, P.Qc, P.Qr, false)) return;  // M Q
    if (!orthonormalize(c, P.Qr, false, ps)) return;
    if (!apply(c, P.Qr, P.Qc, true)) return;   // M^T Q
    if (!orthonormalize(c, P.Qc, false, ps)) return;
  }
  if (!apply(c, P.Qc, P.Qr, false)) return;
  if (!orthonormalize(c, P.Qr, false, ps)) return;
  if (!apply(c, P.Qr, P.Qc, true)) return;  // B^T = M^T Q
  if (!orthonormalize(c, P.Qc, true, ps)) return;
  // every row of both blocks is final; member 0 alone finishes (the others
  // take the next item instead of waiting through the FP64 Jacobi)
  if (!team_meet(c)) return;
  if (member != 0) return;
  rayleigh_ritz(c, P.Racc[ps.racc_cur]);
  __syncthreads();
  // U = Q Vo_k, V = Qt Uo_k over all rows
  c.r0 = 0;
  c.r1 = P.n;
  const int k = P.k;
  for (int idx = threadIdx.x; idx < P.l * P.ld; idx += kThreads) {
    const int i = idx / P.ld, col = idx - i * P.ld;
    sm.B[idx] = col < k ? __ldcg(P.Lk + (size_t)i * k + col) : 0.f;
  }
  rows_times_small(c, P.Qr, sm.B, P.ld, k, false, P.U, k);
  __syncthreads();
  for (int idx = threadIdx.x; idx < P.l * P.ld; idx += kThreads) {
    const int i = idx / P.ld, col = idx - i * P.ld;
    sm.B[idx] = col < k ? __ldcg(P.Rk + (size_t)i * k + col) : 0.f;
  }
  rows_times_small(c, P.Qc, sm.B, P.ld, k, false, P.V, k);
}

__global__ void __launch_bounds__(kThreads, 1)
    batched_persistent_kernel(const Problem *__restrict__ probs, const Item *__restrict__ items, int32_t n_items,
                              int32_t *next, int32_t max_l, uint32_t spin, int32_t phantom) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int s_item;
  __shared__ Problem sp;  // this item's problem, read once
  const int ldmax = (max_l + 3) & ~3;
  Smem sm;
  sm.W = reinterpret_cast<double *>(smraw);
  sm.vec = sm.W + w_doubles(max_l);
  sm.B = reinterpret_cast<float *>(sm.vec + vec_doubles(max_l));
  sm.stage = sm.B + (size_t)max_l * ldmax;
  sm.ones = sm.stage + stage_floats(ldmax);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const Item item = items[it];
    if (threadIdx.x == 0) sp = probs[item.problem];
    __syncthreads();
    run_member(sp, item.member, spin, phantom, sm);
  }
}

size_t problem_bytes(int64_t n, int32_t l, int32_t ld, int32_t k, int32_t team) {
  size_t off = 0;
  auto take = [&](size_t b) { off += (size_t)round_up((int64_t)b, 256); };
  for (int i = 0; i < 4; ++i) take(sizeof(float) * (size_t)n * ld);  // Qr, Qc, Z1, Z2
  take(sizeof(double) * 2 * (size_t)team * l * l);                   // Gram partials
  take(sizeof(double) * (size_t)team * l);                           // column-sum partials
  take(sizeof(double) * (size_t)l * l);
  take(sizeof(double) * (size_t)l * l);  // Racc x2
  take(sizeof(float) * (size_t)l * k);
  take(sizeof(float) * (size_t)l * k);   // Lk, Rk
  return off;
}

}  // namespace
}  // namespace isvd

using namespace isvd;

extern "C" {

isvd_status isvd_svd_batched_persistent(isvd_operator *const *ops, const int32_t *k, int32_t count, int32_t oversample,
                                        int32_t iters, uint64_t seed, float *const *U, float *const *S,
                                        float *const *V, isvd_info *dev_info, const isvd_persistent_options *opt,
                                        void *stream) {
  if (!ops || !k || !U || !S || !V || count < 1) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument or count < 1");
  if (oversample < 0 || iters < 0) return fail(ISVD_ERR_INVALID_ARGUMENT, "need oversample >= 0, iters >= 0");
  const int32_t max_team = opt && opt->max_team > 0 ? std::min(opt->max_team, kMaxTeam) : kMaxTeam;
  const int64_t team_rows = opt && opt->rows_per_member > 0 ? opt->rows_per_member : kDefaultTeamRows;
  const uint32_t spin = opt && opt->spin_limit > 0 ? (uint32_t)opt->spin_limit : kDefaultSpin;
  const int32_t phantom = opt && opt->test_phantom ? 1 : 0;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0, coop = 0;
  ISVD_CUDA_TRY(cudaGetDevice(&dev));
  ISVD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  ISVD_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return fail(ISVD_ERR_UNSUPPORTED, "the device has no cooperative launch");
  std::vector<Problem> probs(count);
  int32_t max_l = 1;
  for (int i = 0; i < count; ++i) {
    isvd_operator *op = ops[i];
    if (!op || !U[i] || !S[i] || !V[i]) return fail(ISVD_ERR_INVALID_ARGUMENT, "problem %d: null argument", i);
    for (int j = 0; j < i; ++j)
      if (ops[j] == op) return fail(ISVD_ERR_INVALID_ARGUMENT, "problem %d repeats an operator", i);
    const isvd_operator_desc &d = op->desc;
    if (op->compose >= 0 || d.form != ISVD_FORM_POLY || d.A.values || d.adj_coeff != 0.0 || d.lr_rank != 0 ||
        d.gather_rows || d.degree < 1 || op->rows != op->cols)
      return fail(ISVD_ERR_UNSUPPORTED,
                  "problem %d: the persistent form takes polynomial operators of an unweighted graph with at most "
                  "the all-ones term",
                  i);
    const int64_t l = (int64_t)k[i] + oversample;
    if (k[i] < 1) return fail(ISVD_ERR_INVALID_ARGUMENT, "problem %d: k < 1", i);
    if (l > kMaxL) return fail(ISVD_ERR_UNSUPPORTED, "problem %d: k + oversample > %d", i, kMaxL);
    if (l > op->n) return fail(ISVD_ERR_SHAPE, "problem %d: k + oversample exceeds n", i);
    Problem &P = probs[i];
    P.n = (int32_t)op->n;
    P.l = (int32_t)l;
    P.ld = (int32_t)round_up(l, 4);
    P.k = k[i];
    P.team = (int32_t)std::min<int64_t>(std::max<int64_t>(1, ceil_div(op->n, team_rows)), max_team);
    P.team = std::min(P.team, std::max(1, sms));
    P.norm = d.norm;
    P.degree = d.degree;
    P.iters = iters;
    for (int t = 0; t < ISVD_MAX_DEGREE; ++t) P.coeff[t] = t < d.degree ? (float)op->coeffs[t] : 0.f;
    P.ones = (float)d.ones_coeff;
    P.seed = seed + (uint64_t)i;
    P.rowptr = d.A.rowptr;
    P.colidx = d.A.colidx;
    P.inv_d = op->inv_d;
    P.s = op->s;
    P.U = U[i];
    P.S = S[i];
    P.V = V[i];
    max_l = std::max(max_l, P.l);
  }
  // workspace: each problem in its own operator's arena; the table and the
  // queue after problem 0's buffers
  std::vector<Item> items;
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  auto cost = [&](int i) { return (double)probs[i].n * probs[i].l * (probs[i].l + 8.0 * probs[i].degree); };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  for (int i : order)
    for (int m = 0; m < probs[i].team; ++m) items.push_back(Item{i, m});
  // table (in operator 0's arena, after its problem): problems, items, then
  // one zeroed region: the queue counter, per problem [arrive, abandoned], infos
  const size_t probs_bytes = (size_t)round_up((int64_t)(sizeof(Problem) * count), 256);
  const size_t items_bytes = (size_t)round_up((int64_t)(sizeof(Item) * items.size()), 256);
  const size_t zero_bytes = 256 + (size_t)round_up((int64_t)(2 * sizeof(int32_t) * count), 256) +
                            sizeof(isvd_info) * (size_t)count;
  const size_t table_bytes = probs_bytes + items_bytes + zero_bytes;
  for (int i = 0; i < count; ++i) {
    Problem &P = probs[i];
    const size_t need = problem_bytes(P.n, P.l, P.ld, P.k, P.team) + (i == 0 ? table_bytes : 0);
    ISVD_TRY(ensure_arena(ops[i], need, s));
    char *base = (char *)ops[i]->arena;
    size_t off = 0;
    auto take = [&](size_t b) {
      char *p = base + off;
      off += (size_t)round_up((int64_t)b, 256);
      return p;
    };
    P.Qr = (float *)take(sizeof(float) * (size_t)P.n * P.ld);
    P.Qc = (float *)take(sizeof(float) * (size_t)P.n * P.ld);
    P.Z1 = (float *)take(sizeof(float) * (size_t)P.n * P.ld);
    P.Z2 = (float *)take(sizeof(float) * (size_t)P.n * P.ld);
    P.part = (double *)take(sizeof(double) * 2 * (size_t)P.team * P.l * P.l);
    P.csum = (double *)take(sizeof(double) * (size_t)P.team * P.l);
    P.Racc[0] = (double *)take(sizeof(double) * (size_t)P.l * P.l);
    P.Racc[1] = (double *)take(sizeof(double) * (size_t)P.l * P.l);
    P.Lk = (float *)take(sizeof(float) * (size_t)P.l * P.k);
    P.Rk = (float *)take(sizeof(float) * (size_t)P.l * P.k);
  }
  char *tb = (char *)ops[0]->arena + problem_bytes(probs[0].n, probs[0].l, probs[0].ld, probs[0].k, probs[0].team);
  Problem *d_probs = (Problem *)tb;
  Item *d_items = (Item *)(tb + probs_bytes);
  char *zero = tb + probs_bytes + items_bytes;
  int32_t *d_next = (int32_t *)zero;
  int32_t *flags = (int32_t *)(zero + 256);
  isvd_info *own = (isvd_info *)(zero + 256 + round_up((int64_t)(2 * sizeof(int32_t) * count), 256));
  for (int i = 0; i < count; ++i) {
    probs[i].arrive = (unsigned *)(flags + 2 * i);
    probs[i].err = flags + 2 * i + 1;
    probs[i].info = dev_info ? dev_info + i : own + i;
  }
  ISVD_CUDA_TRY(cudaMemsetAsync(zero, 0, zero_bytes, s));
  if (dev_info) ISVD_CUDA_TRY(cudaMemsetAsync(dev_info, 0, sizeof(isvd_info) * count, s));
  ISVD_CUDA_TRY(cudaMemcpyAsync(d_probs, probs.data(), sizeof(Problem) * count, cudaMemcpyHostToDevice, s));
  ISVD_CUDA_TRY(cudaMemcpyAsync(d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice, s));
  const size_t smem = smem_bytes(max_l, (max_l + 3) & ~3);
  ISVD_CUDA_TRY(cudaFuncSetAttribute(batched_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  ISVD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_persistent_kernel, kThreads, smem));
  if (per_sm < 1) return fail(ISVD_ERR_UNSUPPORTED, "the persistent kernel does not fit an SM");
  const int grid = (int)std::min<int64_t>((int64_t)items.size(), (int64_t)sms * per_sm);
  int biggest_team = 1;
  for (const Problem &P : probs) biggest_team = std::max(biggest_team, P.team);
  if (grid < biggest_team + phantom && grid < (int)items.size())
    return fail(ISVD_ERR_UNSUPPORTED, "too few resident CTAs for a team");
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  ISVD_CUDA_TRY(cudaLaunchKernelEx(&cfg, batched_persistent_kernel, (const Problem *)d_probs, (const Item *)d_items,
                                   (int32_t)items.size(), d_next, max_l, spin, phantom));
  return ISVD_OK;
}

}  // extern "C"
