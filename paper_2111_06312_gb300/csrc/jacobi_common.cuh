// Device helpers of the one-sided Jacobi SVD (the Rayleigh-Ritz step of
// Alg. 1), shared by the cluster and grid forms (jacobi.cu) and the
// persistent batched kernel.
#pragma once

#include <cstdint>

namespace isvd {
namespace {

// The rotation of a pair with g_p.g_q = ga and squared norms al, be, or
// false when the pair counts as orthogonal: ga^2 <= tol^2 al be (no square
// root: an FP64 square root costs ~10 times an FMA on this part, and an FP64
// instruction ~64 clocks of a warp).  The tangent t (Rutishauser) is taken in
// FP32 from zeta = (be - al) / (2 ga) scaled by a power of two: it only sets
// how far the pair turns, so an FP32-accurate t leaves g_p.g_q at ~1e-7 of its
// size (cleared in the next sweep) but cannot cost accuracy; cs = (1 + t^2)^-1/2
// and sn = t cs in FP64 keep the rotation orthogonal to FP64 rounding.
__device__ __forceinline__ bool jacobi_angle(double ga, double al, double be, double tol, double tiny, double &t,
                                             double &cs, double &sn) {
  if (ga == 0.0 || ga * ga <= (tol * tol) * (al * be)) return false;
  if (al <= tiny && be <= tiny) return false;
  const double num = be - al, den = 2.0 * ga;
  const int e = ((__double2hiint(den) >> 20) & 0x7FF) - 1023;  // den = 2^e (1 + f)
  const double sc = __hiloint2double((1023 - e) << 20, 0);    // 2^-e
  const float zf = __double2float_rn(num * sc) / __double2float_rn(den * sc);
  float tf;
  if (fabsf(zf) < 1e18f)
    tf = copysignf(1.f, zf) / (fabsf(zf) + sqrtf(fmaf(zf, zf, 1.f)));
  else
    tf = 0.5f / zf;  // t ~ 1 / (2 zeta); 0 when zeta overflowed
  t = (double)tf;
  cs = rsqrt(fma(t, t, 1.0));
  sn = cs * t;
  return true;
}

// round-robin tournament on m (even) players: round r, pair k
__device__ __forceinline__ void tourney(int r, int k, int m, int &p, int &q) {
  if (k == 0) {
    p = r;
    q = m - 1;
  } else {
    p = (r + k) % (m - 1);
    q = (r - k + (m - 1)) % (m - 1);
  }
}

// Descending order of the first l column norms (the rest are zero padding),
// stable: rank of column p = #columns with a larger norm, or an equal norm
// and a smaller index (a NaN norm ranks below every number).  One CTA.
__device__ void jacobi_order(const double *nrm_g, int l, int32_t *perm_g) {
  __shared__ double snrm[ISVD_MAX_BLOCK_WIDE];
  for (int p = threadIdx.x; p < l; p += blockDim.x) {
    const double x = __ldcg(nrm_g + p);
    snrm[p] = x == x ? x : -1.0;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < l; p += blockDim.x) {
    const double x = snrm[p];
    int rank = 0;
    for (int q = 0; q < l; ++q) rank += (snrm[q] > x || (snrm[q] == x && q < p)) ? 1 : 0;
    perm_g[rank] = p;
  }
}

// Column kk = first, first + stride, ... of Vo = w_p / sigma and of
// Uo = A w_p / sigma^2 (p = perm[kk]); w_p is staged in shared memory (wsm,
// l doubles), one warp per row of A (coalesced).
__device__ void jacobi_outputs(const double *__restrict__ A, int l, const double *Wg, const double *nrm_g,
                               const int32_t *perm_g, int first, int stride, double *wsm, double *__restrict__ Uo,
                               double *__restrict__ S, double *__restrict__ Vo, float *__restrict__ Uk,
                               float *__restrict__ Vk, float *__restrict__ Sk, int32_t k) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  for (int kk = first; kk < l; kk += stride) {
    const int p = __ldcg(perm_g + kk);
    const double sg = __ldcg(nrm_g + p);
    __syncthreads();  // the previous column's readers are done
    for (int i = tid; i < l; i += blockDim.x) wsm[i] = __ldcg(Wg + (size_t)p * l + i);
    __syncthreads();
    const bool need_u = Uo || (Uk && kk < k);
    for (int i = warp; i < l; i += nwarp) {
      double u = 0.0;
      if (need_u) {
        for (int t = lane; t < l; t += 32) u += A[(size_t)i * l + t] * wsm[t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
      }
      if (lane == 0) {
        const double v = sg > 0.0 ? wsm[i] / sg : 0.0;
        u = sg > 0.0 ? u / (sg * sg) : 0.0;
        if (Vo) Vo[(size_t)i * l + kk] = v;
        if (Uo) Uo[(size_t)i * l + kk] = u;
        if (kk < k) {
          if (Vk) Vk[(size_t)i * k + kk] = (float)v;
          if (Uk) Uk[(size_t)i * k + kk] = (float)u;
        }
      }
    }
    if (tid == 0) {
      if (S) S[kk] = sg;
      if (Sk && kk < k) Sk[kk] = (float)sg;
    }
  }
}

// ||A||_F^2 by every CTA (the same value everywhere)
__device__ double frobenius2(const double *A, int l, double *red) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  double f = 0.0;
  for (int idx = tid; idx < l * l; idx += blockDim.x) f += A[idx] * A[idx];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
  if (lane == 0) red[warp] = f;
  __syncthreads();
  double fro2 = 0.0;
  for (int w = 0; w < nwarp; ++w) fro2 += red[w];
  return fro2;
}

}  // namespace
}  // namespace isvd
