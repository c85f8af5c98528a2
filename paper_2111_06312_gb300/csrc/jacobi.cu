// Small SVD of the Rayleigh-Ritz step (Alg. 1): A = Uo diag(S) Vo^T for an
// l x l FP64 matrix (A = R from the QR of B^T), by one-sided Jacobi on the
// columns of G = A^T, spread over a thread-block cluster.
//
// GB300 runs FP64 at ~8 GFLOP/s per SM, so one CTA cannot do the ~5 l^3 flop
// per sweep quickly; the columns are split into 2*CL blocks held in the
// shared memory of the CL CTAs of one cluster.  A sweep rotates every column
// pair once: the pairs inside each block first, then the pairs across blocks,
// block pairs meeting in round-robin tournament order with the blocks
// travelling between CTAs through distributed shared memory (one cluster
// barrier per step).  Rotations are not accumulated: after convergence the
// columns w_p of G J have norms sigma_p, Vo = W Sigma^-1 and
// Uo = J = A W Sigma^-2 (A A^T j_p = sigma_p^2 j_p), one FP64 product.
// Rotation: Rutishauser's formula, column norms carried along (recomputed each
// sweep); converged when every pair satisfies |g_p.g_q| <= tol ||g_p|| ||g_q||,
// tol = max(1e-15, sqrt(l) eps).
//
// Wide blocks (l > 160) run the same sweeps over a whole grid instead
// (`jacobi_grid_kernel`): the FP64 work grows as l^3 and one cluster's 16 SMs
// hold only a tenth of the GPU's FP64 units.  The columns then stay in global
// memory (L2-resident: 2 MB at l = 512) at fixed places, blocks of two columns,
// one CTA per block pair of the tournament step; a step moves no data, and
// the steps are separated by a grid barrier (cooperative launch, bounded
// waits).  Every read of a column goes to L2 (ld.global.cg) so that no CTA
// reads a stale L1 copy of a column another CTA has rotated since.  The
// cluster kernel keeps this global-memory form as well, for blocks beyond its
// shared memory where a cooperative launch is not available.
#include <cooperative_groups.h>

#include <mutex>

#include "internal.h"
#include "jacobi_common.cuh"

namespace cg = cooperative_groups;

namespace isvd {
namespace {

constexpr int kJacThreads = 256;
constexpr int kJacMaxCluster = 16;
constexpr int kJacMaxSmem = 200 * 1024;

// One warp rotates columns gp, gq (length l, squared norms *np, *nq kept by the
// caller) if they are not yet orthogonal.  Only g_p . g_q is summed; the norms
// follow the rotation in closed form (||g_p'||^2 = ||g_p||^2 - t g_p.g_q,
// ||g_q'||^2 = ||g_q||^2 + t g_p.g_q) and are recomputed exactly every sweep.
// a column element: from shared memory, or (global mode) from L2
__device__ __forceinline__ double ldc(const double *p, bool gmode) { return gmode ? __ldcg(p) : *p; }

__device__ __forceinline__ int rotate_pair(double *gp, double *gq, double *np, double *nq, int l, int lane,
                                           double tol, double tiny, bool gmode) {
  double ga = 0.0;
  for (int i = lane; i < l; i += 32) ga += ldc(gp + i, gmode) * ldc(gq + i, gmode);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
  const double al = ldc(np, gmode), be = ldc(nq, gmode);
  double t, cs, sn;
  if (!jacobi_angle(ga, al, be, tol, tiny, t, cs, sn)) return 0;
  for (int i = lane; i < l; i += 32) {
    const double x = ldc(gp + i, gmode), y = ldc(gq + i, gmode);
    gp[i] = cs * x - sn * y;
    gq[i] = sn * x + cs * y;
  }
  __syncwarp();
  if (lane == 0) {
    *np = al - t * ga;
    *nq = be + t * ga;
  }
  __syncwarp();
  return 1;
}

__global__ void __launch_bounds__(kJacThreads) jacobi_cluster_kernel(
    const double *__restrict__ A, int32_t l, int32_t bs, double *__restrict__ Wg, double *__restrict__ nrm_g,
    int32_t *__restrict__ perm_g, double *__restrict__ Uo, double *__restrict__ S, double *__restrict__ Vo,
    float *__restrict__ Uk, float *__restrict__ Vk, float *__restrict__ Sk, int32_t k, isvd_info *info,
    int32_t iters, int32_t gmode, double *__restrict__ gnrm) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int c = (int)cluster.block_rank();
  const int nb = 2 * CL;
  const int l3 = nb * bs;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  extern __shared__ double sm[];  // [2 buffers][2 slots][bs][l], then norms [2 buffers][2 slots][bs]
  __shared__ int ids[2][2];
  __shared__ int any_flags[kJacMaxCluster];
  __shared__ int stop;
  __shared__ double red[kJacThreads / 32];
  // shared-memory mode: [2 buffers][2 slots][bs][l] then the norms; global
  // mode: block b's columns at Wg[b bs ..] and norms at gnrm[b bs ..]
  const bool gm = gmode != 0;
  auto colp = [&](int buf, int slot, int j) {
    return gm ? Wg + ((size_t)ids[buf][slot] * bs + j) * l : sm + ((size_t)(buf * 2 + slot) * bs + j) * l;
  };
  double *nrm = sm + (size_t)4 * bs * l;
  auto nrmp = [&](int buf, int slot, int j) {
    return gm ? gnrm + (size_t)ids[buf][slot] * bs + j : nrm + (buf * 2 + slot) * bs + j;
  };

  if (tid == 0) {
    ids[0][0] = c;
    ids[0][1] = nb - 1 - c;
  }
  __syncthreads();
  for (int slot = 0; slot < 2; ++slot)
    for (int idx = tid; idx < bs * l; idx += blockDim.x) {
      const int j = idx / l, i = idx - j * l;
      const int p = ids[0][slot] * bs + j;
      colp(0, slot, j)[i] = (p < l) ? A[(size_t)p * l + i] : 0.0;
    }
  const double fro2 = frobenius2(A, l, red);
  const double eps = 2.220446049250313e-16;
  const double tol = fmax(1e-15, sqrt((double)l) * eps);
  const double tiny = (double)l * eps * (double)l * eps * fro2;
  const int bsp = (bs + 1) & ~1;  // players of the in-block tournament
  int cur = 0, sweeps = 0;
  cluster.sync();
  for (int sweep = 0; sweep < 60; ++sweep) {
    int rotated = 0;
    sweeps = sweep + 1;
    // exact squared norms of the columns held here
    for (int q = warp; q < 2 * bs; q += nwarp) {
      const double *g = colp(cur, q / bs, q % bs);
      double s2 = 0.0;
      for (int i = lane; i < l; i += 32) {
        const double x = ldc(g + i, gm);
        s2 += x * x;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) *nrmp(cur, q / bs, q % bs) = s2;
    }
    __syncthreads();
    // pairs inside each of the two blocks held here
    for (int r = 0; r < bsp - 1; ++r) {
      for (int pi = warp; pi < bsp; pi += nwarp) {  // bsp/2 pairs per slot, two slots
        const int slot = pi / (bsp / 2), kk = pi - slot * (bsp / 2);
        int p, q;
        tourney(r, kk, bsp, p, q);
        if (p < bs && q < bs)
          rotated |= rotate_pair(colp(cur, slot, p), colp(cur, slot, q), nrmp(cur, slot, p), nrmp(cur, slot, q), l,
                                 lane, tol, tiny, gm);
      }
      __syncthreads();
    }
    // pairs across blocks: nb - 1 tournament steps
    for (int step = 0; step < nb - 1; ++step) {
      for (int r = 0; r < bs; ++r) {
        for (int i = warp; i < bs; i += nwarp)
          rotated |= rotate_pair(colp(cur, 0, i), colp(cur, 1, (i + r) % bs), nrmp(cur, 0, i),
                                 nrmp(cur, 1, (i + r) % bs), l, lane, tol, tiny, gm);
        __syncthreads();
      }
      if (CL == 1) continue;  // two blocks only: they never move
      if (gm) __threadfence();  // the rotated columns, before other CTAs take the blocks
      cluster.sync();
      // circle [t1 .. t_{CL-1}, b_{CL-1} .. b0] rotates by one; t0 stays
      const int nxt = cur ^ 1;
      int src_rank[2], src_slot[2];
      if (c == 0) {
        src_rank[0] = 0; src_slot[0] = 0;
      } else if (c == 1) {
        src_rank[0] = 0; src_slot[0] = 1;
      } else {
        src_rank[0] = c - 1; src_slot[0] = 0;
      }
      if (c == CL - 1) {
        src_rank[1] = c; src_slot[1] = 0;
      } else {
        src_rank[1] = c + 1; src_slot[1] = 1;
      }
      for (int slot = 0; slot < 2; ++slot) {
        if (!gm) {  // global mode: the blocks stay where they are, only their ids move
          double *src = cluster.map_shared_rank(colp(cur, src_slot[slot], 0), src_rank[slot]);
          double *dst = colp(nxt, slot, 0);
          for (int idx = tid; idx < bs * l; idx += blockDim.x) dst[idx] = src[idx];
          const double *nsrc = cluster.map_shared_rank(nrmp(cur, src_slot[slot], 0), src_rank[slot]);
          for (int j = tid; j < bs; j += blockDim.x) *nrmp(nxt, slot, j) = nsrc[j];
        }
        if (tid == 0) {
          int *rid = cluster.map_shared_rank(&ids[cur][src_slot[slot]], src_rank[slot]);
          ids[nxt][slot] = *rid;
        }
      }
      cur = nxt;
      __syncthreads();
    }
    // convergence: any rotation anywhere in the cluster?
    const int mine = __syncthreads_or(rotated);
    if (tid == 0) *cluster.map_shared_rank(&any_flags[c], 0) = mine;
    cluster.sync();
    if (tid == 0) {
      const int *fl = cluster.map_shared_rank(any_flags, 0);
      int any = 0;
      for (int r = 0; r < CL; ++r) any |= fl[r];
      stop = !any;
    }
    cluster.sync();  // any_flags of CTA 0 are rewritten next sweep
    if (stop) break;
  }
  // columns and norms to global memory, by original block position
  for (int slot = 0; slot < 2; ++slot)
    for (int j = warp; j < bs; j += nwarp) {
      const int p = ids[cur][slot] * bs + j;
      const double *g = colp(cur, slot, j);
      double s2 = 0.0;
      for (int i = lane; i < l; i += 32) {
        const double x = ldc(g + i, gm);
        s2 += x * x;
        if (!gm) Wg[(size_t)p * l + i] = x;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) nrm_g[p] = sqrt(s2);
    }
  __threadfence();
  cluster.sync();
  if (c == 0) {
    jacobi_order(nrm_g, l, perm_g);
    if (tid == 0 && info) info->iters_done = iters >= 0 ? iters : sweeps;
  }
  (void)l3;
  __threadfence();
  cluster.sync();
  // outputs (no CTA reads another's shared memory any more)
  jacobi_outputs(A, l, Wg, nrm_g, perm_g, c, CL, sm, Uo, S, Vo, Uk, Vk, Sk, k);
}

// ---- the grid form (wide blocks) ---------------------------------------------------
struct GridBar {
  unsigned count, gen;
  int err;
  int any[2];  // a rotation happened in the sweep (even, odd sweeps)
  int pad[3];
};
constexpr size_t kGridBarDoubles = (sizeof(GridBar) + 7) / 8;
constexpr uint32_t kGridSpinLimit = 1u << 22;  // ~1 s of short sleeps: far beyond any step

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void group_sync(int id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }

// A wait of thread 0 gave up: flag it for every CTA, report TIMEOUT.
__device__ void give_up(GridBar *b, isvd_info *info) {
  atomicExch(&b->err, 1);
  if (info) atomicExch(&info->status, (int)ISVD_ERR_TIMEOUT);
}

// Barrier of all CTAs of a cooperative launch, with a bounded wait: false
// when this CTA gave up (it then sets TIMEOUT and every later wait of any
// CTA gives up at once), so that the kernel ends in bounded time.
__device__ bool grid_sync(GridBar *b, isvd_info *info) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    const unsigned g = *(volatile unsigned *)&b->gen;
    if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      uint32_t spins = 0;
      while (*(volatile unsigned *)&b->gen == g) {
        if (*(volatile int *)&b->err || ++spins > kGridSpinLimit) {
          give_up(b, info);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// Thread 0 waits until both blocks' release counters reach `need`.
__device__ bool wait_blocks(const unsigned *ver, int bp, int bq, unsigned need, GridBar *b, isvd_info *info) {
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = 1;
    uint32_t spins = 0;
    while (ld_acquire(ver + bp) < need || ld_acquire(ver + bq) < need) {
      if (*(volatile int *)&b->err || ++spins > kGridSpinLimit) {
        give_up(b, info);
        ok = 0;
        break;
      }
      __nanosleep(20);
    }
  }
  __syncthreads();
  return ok != 0;
}

// One rotation of columns x, y (shared memory, length l) by a group of four
// warps (gt = thread in the group, gw = warp in the group, named barrier id):
// g_x.g_y summed over the group in a fixed order, so that every thread takes
// the same decision.  Squared norms *nx, *ny as in rotate_pair.
__device__ int rotate_group(double *x, double *y, double *nx, double *ny, int l, int gt, int gw, double *gred, int id,
                            double tol, double tiny) {
  double ga = 0.0;
  for (int i = gt; i < l; i += 128) ga += x[i] * y[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ga += __shfl_xor_sync(0xffffffffu, ga, o);
  if ((gt & 31) == 0) gred[gw] = ga;
  group_sync(id);
  ga = (gred[0] + gred[1]) + (gred[2] + gred[3]);
  const double al = *nx, be = *ny;
  double t, cs, sn;
  const int rot = jacobi_angle(ga, al, be, tol, tiny, t, cs, sn) ? 1 : 0;
  if (rot) {
    for (int i = gt; i < l; i += 128) {
      const double a = x[i], b = y[i];
      x[i] = cs * a - sn * b;
      y[i] = sn * a + cs * b;
    }
    if (gt == 0) {
      *nx = al - t * ga;
      *ny = be + t * ga;
    }
  }
  group_sync(id);  // gred and the norms are read again by the next rotation
  return rot;
}

// Blocks of two columns (Wg row p = column p of G = A^T, zero beyond l),
// nb = 2 gridDim.x of them.  CTA c loads blocks 2c and 2c+1 and rotates the
// pair inside each at the start of a sweep; in tournament step t it takes
// block pair c, waiting only for the two CTAs that released those blocks in
// the step before (per-block release counters; no grid barrier inside a
// sweep).  A step stages the four columns in shared memory; the two groups
// of four warps rotate two disjoint pairs at a time.
__global__ void __launch_bounds__(kJacThreads) jacobi_grid_kernel(
    const double *__restrict__ A, int32_t l, double *__restrict__ Wg, double *__restrict__ nrm_g,
    int32_t *__restrict__ perm_g, double *__restrict__ Uo, double *__restrict__ S, double *__restrict__ Vo,
    float *__restrict__ Uk, float *__restrict__ Vk, float *__restrict__ Sk, int32_t k, isvd_info *info,
    int32_t iters, GridBar *bar, unsigned *ver) {
  const int G = (int)gridDim.x, c = (int)blockIdx.x, nb = 2 * G;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = warp >> 2, gt = tid & 127, gw = warp & 3;
  extern __shared__ double sm[];  // four columns [4][l] (one column of the outputs at the end)
  __shared__ double red[kJacThreads / 32];
  __shared__ double n4[4];
  __shared__ double gred[2][4];
  __shared__ int stop;
  const int own0 = 4 * c;
  for (int idx = tid; idx < 4 * l; idx += blockDim.x) {
    const int j = idx / l, i = idx - j * l;
    const int p = own0 + j;
    Wg[(size_t)p * l + i] = p < l ? A[(size_t)p * l + i] : 0.0;
  }
  const double fro2 = frobenius2(A, l, red);
  const double eps = 2.220446049250313e-16;
  const double tol = fmax(1e-15, sqrt((double)l) * eps);
  const double tiny = (double)l * eps * (double)l * eps * fro2;
  auto col = [&](int j) { return sm + (size_t)j * l; };
  // stage columns p0, p0+1 (slots 0, 1) and q0, q0+1 (slots 2, 3)
  auto load4 = [&](int p0, int q0, bool norms) {
    for (int idx = tid; idx < 4 * l; idx += blockDim.x) {
      const int j = idx / l, i = idx - j * l;
      const int p = (j < 2 ? p0 : q0) + (j & 1);
      sm[idx] = __ldcg(Wg + (size_t)p * l + i);
    }
    if (!norms && tid < 4) n4[tid] = __ldcg(nrm_g + (tid < 2 ? p0 : q0) + (tid & 1));
    __syncthreads();
  };
  auto store4 = [&](int p0, int q0) {
    for (int idx = tid; idx < 4 * l; idx += blockDim.x) {
      const int j = idx / l, i = idx - j * l;
      const int p = (j < 2 ? p0 : q0) + (j & 1);
      Wg[(size_t)p * l + i] = sm[idx];
    }
    if (tid < 4) nrm_g[(tid < 2 ? p0 : q0) + (tid & 1)] = n4[tid];
    __syncthreads();
  };
  auto release = [&](int bp, int bq, unsigned v) {
    if (tid == 0) {
      __threadfence();
      st_release(ver + bp, v);
      st_release(ver + bq, v);
    }
  };
  int sweeps = 0;
  if (!grid_sync(bar, info)) return;
  for (int sweep = 0; sweep < 60; ++sweep) {
    int rotated = 0;
    sweeps = sweep + 1;
    const unsigned base = (unsigned)sweep * (unsigned)nb;
    // own blocks: exact squared norms, then the pair inside each block
    load4(own0, own0 + 2, true);
    if (warp < 4) {
      double s2 = 0.0;
      for (int i = lane; i < l; i += 32) s2 += col(warp)[i] * col(warp)[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) n4[warp] = s2;
    }
    __syncthreads();
    rotated |= rotate_group(col(2 * grp), col(2 * grp + 1), &n4[2 * grp], &n4[2 * grp + 1], l, gt, gw, gred[grp],
                            1 + grp, tol, tiny);
    __syncthreads();
    store4(own0, own0 + 2);
    release(2 * c, 2 * c + 1, base + 1);
    // pairs across blocks: nb - 1 tournament steps, block pair c of each
    for (int step = 0; step < nb - 1; ++step) {
      int bp, bq;
      tourney(step, c, nb, bp, bq);
      if (!wait_blocks(ver, bp, bq, base + 1 + step, bar, info)) return;
      load4(2 * bp, 2 * bq, false);
      // round 0: (p0, q0), (p1, q1); round 1: (p0, q1), (p1, q0)
      rotated |= rotate_group(col(grp), col(2 + grp), &n4[grp], &n4[2 + grp], l, gt, gw, gred[grp], 1 + grp, tol,
                              tiny);
      __syncthreads();
      rotated |= rotate_group(col(grp), col(3 - grp), &n4[grp], &n4[3 - grp], l, gt, gw, gred[grp], 1 + grp, tol,
                              tiny);
      __syncthreads();
      store4(2 * bp, 2 * bq);
      release(bp, bq, base + 2 + step);
    }
    // convergence: any rotation anywhere in the grid?
    const int mine = __syncthreads_or(rotated);
    if (tid == 0 && mine) atomicOr(&bar->any[sweep & 1], 1);
    if (!grid_sync(bar, info)) return;
    if (tid == 0) {
      stop = *(volatile int *)&bar->any[sweep & 1] == 0;
      if (c == 0) bar->any[(sweep + 1) & 1] = 0;  // read by nobody before two more barriers
    }
    __syncthreads();
    if (stop) break;
  }
  for (int q = warp; q < 4; q += kJacThreads / 32) {
    const double *g = Wg + (size_t)(own0 + q) * l;
    double s2 = 0.0;
    for (int i = lane; i < l; i += 32) {
      const double x = __ldcg(g + i);
      s2 += x * x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane == 0) nrm_g[own0 + q] = sqrt(s2);
  }
  if (!grid_sync(bar, info)) return;
  if (c == 0) {
    jacobi_order(nrm_g, l, perm_g);
    if (tid == 0 && info) info->iters_done = iters >= 0 ? iters : sweeps;
  }
  if (!grid_sync(bar, info)) return;
  jacobi_outputs(A, l, Wg, nrm_g, perm_g, c, G, sm, Uo, S, Vo, Uk, Vk, Sk, k);
}

constexpr int kGridBs = 2;  // columns per block of the grid form
constexpr int kGridMinL = ISVD_MAX_BLOCK + 1;  // narrower blocks take the cluster form

int g_cluster = 0;
int g_grid_max = 0;  // CTAs a cooperative launch of the grid form may have (0: none)
std::once_flag g_once;
cudaError_t g_err = cudaSuccess;

size_t jac_smem(int32_t l, int32_t bs) { return sizeof(double) * 4 * (size_t)bs * (l + 1); }
// global mode: shared memory only stages one column of the outputs
size_t jac_smem_global(int32_t l) { return sizeof(double) * (size_t)l; }
// grid form: the four columns of a step
size_t jac_smem_grid(int32_t l) { return sizeof(double) * 4 * (size_t)l; }

int block_size_for(int32_t l, int cl) { return (int)((l + 2 * cl - 1) / (2 * cl)); }

cudaError_t pick_cluster() {
  std::call_once(g_once, [] {
    cudaError_t e = cudaFuncSetAttribute(jacobi_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) cudaGetLastError();
    e = cudaFuncSetAttribute(jacobi_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kJacMaxSmem);
    if (e != cudaSuccess) {
      g_err = e;
      return;
    }
    // the grid form: a cooperative launch of up to one CTA per SM
    int dev = 0, coop = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && coop &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_grid_kernel, kJacThreads,
                                                      jac_smem_grid(ISVD_MAX_BLOCK_WIDE)) == cudaSuccess)
      g_grid_max = sms * per_sm;
    else
      cudaGetLastError();
    g_cluster = 1;
    for (int cl : {16, 8, 4, 2}) {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(cl);
      cfg.blockDim = dim3(kJacThreads);
      cfg.dynamicSmemBytes = jac_smem(ISVD_MAX_BLOCK, block_size_for(ISVD_MAX_BLOCK, cl));
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cl;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, jacobi_cluster_kernel, &cfg) == cudaSuccess && nclusters > 0) {
        g_cluster = cl;
        break;
      }
      cudaGetLastError();
    }
  });
  return g_err;
}

}  // namespace

int grid_ctas(int32_t l) { return (int)((l + 2 * kGridBs - 1) / (2 * kGridBs)); }

cudaError_t small_svd_launch(const double *A, int32_t l, double *Uo, double *S, double *Vo, double *work, float *Uk,
                             float *Vk, float *Sk, int32_t k, isvd_info *info, int32_t iters, cudaStream_t s) {
  cudaError_t e = pick_cluster();
  if (e != cudaSuccess) return e;
  if (l >= kGridMinL && grid_ctas(l) <= g_grid_max) {
    const int G = grid_ctas(l);
    const int l3 = 2 * G * kGridBs;
    double *Wg = work;                                      // l3 x l
    double *nrm = work + (size_t)l3 * l;                    // l3
    int32_t *perm = reinterpret_cast<int32_t *>(nrm + l3);  // l
    GridBar *bar = reinterpret_cast<GridBar *>(nrm + l3 + (l + 1) / 2 + 1);
    unsigned *ver = reinterpret_cast<unsigned *>(bar + 1);  // 2 G block release counters
    e = cudaMemsetAsync(bar, 0, sizeof(GridBar) + sizeof(unsigned) * 2 * G, s);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kJacThreads);
    cfg.dynamicSmemBytes = jac_smem_grid(l);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, jacobi_grid_kernel, A, l, Wg, nrm, perm, Uo, S, Vo, Uk, Vk, Sk, k, info, iters,
                              bar, ver);
  }
  // at least 4 columns per block (fewer CTAs for small l)
  int cl = g_cluster;
  while (cl > 1 && block_size_for(l, cl) < 4) cl >>= 1;
  const int bs = block_size_for(l, cl);
  const int l3 = 2 * cl * bs;
  if (l > ISVD_MAX_BLOCK_WIDE) return cudaErrorInvalidValue;
  // blocks that do not fit the cluster's shared memory stay in global memory
  const int32_t gmode = jac_smem(l, bs) > (size_t)kJacMaxSmem ? 1 : 0;
  double *Wg = work;                                   // l3 x l
  double *nrm = work + (size_t)l3 * l;                 // l3 (squared norms during the sweeps in global mode)
  int32_t *perm = reinterpret_cast<int32_t *>(nrm + l3);  // l
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(kJacThreads);
  cfg.dynamicSmemBytes = gmode ? jac_smem_global(l) : jac_smem(l, bs);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel, A, l, bs, Wg, nrm, perm, Uo, S, Vo, Uk, Vk, Sk, k, info,
                            iters, gmode, nrm);
}

size_t small_svd_work_doubles(int32_t l) {
  // largest l3 over the cluster sizes and the grid form, plus norms, order
  // and the grid barrier
  size_t best = 0;
  auto need = [&](size_t l3) {
    const size_t x = l3 * l + l3 + (l + 1) / 2 + 1 + kGridBarDoubles + l3 / 2;  // l3 / 2 >= counters
    if (x > best) best = x;
  };
  for (int cl = 1; cl <= kJacMaxCluster; cl <<= 1) need((size_t)2 * cl * block_size_for(l, cl));
  need((size_t)2 * grid_ctas(l) * kGridBs);
  return best;
}

}  // namespace isvd
