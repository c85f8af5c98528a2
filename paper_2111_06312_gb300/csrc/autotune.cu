// Launch-shape autotuner for the sparse products, and the failure-detection
// self-test of the bounded waits.
//
// The autotuner times isvd_apply on the operator, at the caller's block width
// and storage type, for a fixed list of launch shapes (row kernel variants:
// occupancy, L2 budget for hub columns, hub split threshold, wide slabs,
// packed temporaries; the ring kernel; the packed-slab kernel at three slab
// widths) and keeps the fastest.  Results can be kept
// in a text cache keyed by the operator's shape, its degree histogram, the
// block width, the storage type and the device name, so that a later process
// skips the timing.  The paper has no counterpart (it called library kernels).
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "tc_common.cuh"

namespace isvd {
namespace {

__global__ void wait_selftest_kernel(int32_t limit, isvd_info *info) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  // nothing arrives on the barrier: the wait must give up and report
  if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, limit)) atomicExch(&info->status, (int)ISVD_ERR_TIMEOUT);
}

uint64_t fnv1a(const void *p, size_t n, uint64_t h = 1469598103934665603ull) {
  const unsigned char *c = static_cast<const unsigned char *>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

std::string tune_key(const isvd_operator *op, int32_t b, isvd_dtype dtype) {
  cudaDeviceProp prop{};
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  std::string name(prop.name);
  for (char &ch : name)
    if (ch == ' ' || ch == '|') ch = '_';
  const uint64_t h = fnv1a(op->tags_A.hist, sizeof op->tags_A.hist);
  char buf[512];
  snprintf(buf, sizeof buf, "rows=%lld cols=%lld nnz=%lld xnnz=%lld form=%d norm=%d deg=%d L=%d b=%d dt=%d hist=%016llx dev=%s",
           (long long)op->rows, (long long)op->cols, (long long)op->desc.A.nnz, (long long)op->x_nnz,
           (int)op->desc.form, (int)op->desc.norm, op->desc.degree, op->desc.L, b, (int)dtype,
           (unsigned long long)h, name.c_str());
  return buf;
}

bool cache_lookup(const char *path, const std::string &key, isvd_tuning *t) {
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    char *bar = strchr(line, '|');
    if (!bar) continue;
    *bar = 0;
    if (key != line) continue;
    isvd_tuning x{};
    if (sscanf(bar + 1, "%d %d %d %d %d %d %d", &x.slab_cols_f32, &x.slab_cols_bf16, &x.heavy_threshold,
               &x.heavy_chunk, &x.flags, &x.chunk_nnz, &x.l2_budget_mb) == 7) {
      *t = x;  // the last matching line wins
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char *path, const std::string &key, const isvd_tuning &t) {
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s|%d %d %d %d %d %d %d\n", key.c_str(), t.slab_cols_f32, t.slab_cols_bf16, t.heavy_threshold,
          t.heavy_chunk, t.flags, t.chunk_nnz, t.l2_budget_mb);
  fclose(f);
}

}  // namespace
}  // namespace isvd

using namespace isvd;

extern "C" {

isvd_status isvd_selftest_wait(int32_t spin_limit, isvd_info *dev_info, void *stream) {
  if (!dev_info || spin_limit < 1 || spin_limit > (1 << 24))
    return fail(ISVD_ERR_INVALID_ARGUMENT, "need dev_info and 1 <= spin_limit <= 2^24");
  wait_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(spin_limit, dev_info);
  ISVD_CUDA_TRY(cudaGetLastError());
  return ISVD_OK;
}

isvd_status isvd_autotune(isvd_operator *op, int32_t b, isvd_dtype dtype, const char *cache_path, isvd_tuning *out,
                          void *stream) {
  if (!op) return fail(ISVD_ERR_INVALID_ARGUMENT, "null operator");
  if (op->compose >= 0) return fail(ISVD_ERR_UNSUPPORTED, "a composite operator has no launch shapes: tune its children");
  if (b < 1 || b > ISVD_MAX_BLOCK) return fail(ISVD_ERR_INVALID_ARGUMENT, "block width must be in 1..%d", ISVD_MAX_BLOCK);
  if (dtype != ISVD_F32 && dtype != ISVD_BF16) return fail(ISVD_ERR_INVALID_ARGUMENT, "unknown dtype");
  cudaStream_t s = (cudaStream_t)stream;
  const std::string key = tune_key(op, b, dtype);
  isvd_tuning best{};
  if (cache_path && cache_lookup(cache_path, key, &best)) {
    ISVD_TRY(isvd_set_tuning(op, &best, stream));
    if (out) *out = best;
    return ISVD_OK;
  }
  isvd_tuning base{};
  ISVD_TRY(isvd_get_tuning(op, &base));
  std::vector<isvd_tuning> cands;
  auto add = [&](isvd_tuning t) { cands.push_back(t); };
  const int hints = ISVD_TUNE_CACHE_HINTS | ISVD_TUNE_HOT_TAGS;
  isvd_tuning r{128, 256, 128, 128, ISVD_TUNE_ROW_KERNEL | hints | ISVD_TUNE_ROWS_OCC3, 512, 64};
  add(r);
  {
    isvd_tuning t = r;
    t.flags &= ~ISVD_TUNE_ROWS_OCC3;
    add(t);
  }
  for (int mb : {32, 96}) {
    isvd_tuning t = r;
    t.l2_budget_mb = mb;
    add(t);
  }
  {
    isvd_tuning t = r;
    t.flags &= ~ISVD_TUNE_HOT_TAGS;
    add(t);
  }
  for (int ht : {64, 256}) {
    isvd_tuning t = r;
    t.heavy_threshold = t.heavy_chunk = ht;
    add(t);
  }
  {
    isvd_tuning t = r;
    t.slab_cols_f32 = 256;
    t.slab_cols_bf16 = 512;
    add(t);
  }
  {
    isvd_tuning t = r;
    t.flags = ISVD_TUNE_RING_KERNEL | ISVD_TUNE_CACHE_HINTS | ISVD_TUNE_HOT_TAGS;
    add(t);
  }
  {
    isvd_tuning t = r;
    t.flags |= ISVD_TUNE_PACKED;
    add(t);
  }
  // packed slabs of 128, 256 and 512 bytes per row
  for (int w : {32, 64, 128}) {
    isvd_tuning t = r;
    t.flags = ISVD_TUNE_SLAB_KERNEL;
    t.slab_cols_f32 = w;
    t.slab_cols_bf16 = 2 * w;
    add(t);
  }

  // probe blocks: G (cols x ld) from the start-block generator, out (rows x ld)
  const int64_t ld = round_up(b, 8);
  const size_t es = dtype == ISVD_F32 ? 4 : 2;
  void *G = op_alloc(op, es * (size_t)op->cols * ld, s);
  void *Y = op_alloc(op, es * (size_t)op->rows * ld, s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  isvd_status st = ISVD_OK;
  float best_ms = 1e30f;
  if (!G || !Y) {
    st = fail(ISVD_ERR_WORKSPACE, "autotune probe allocation failed");
  } else if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = fail(ISVD_ERR_CUDA, "event creation failed");
  } else {
    const cudaError_t ge = gaussian_launch(12345, op->cols, b, G, ld, dtype == ISVD_F32 ? DT_F32 : DT_BF16, s);
    if (ge != cudaSuccess) st = fail(ISVD_ERR_CUDA, "probe block: %s", cudaGetErrorString(ge));
    for (size_t i = 0; st == ISVD_OK && i < cands.size(); ++i) {
      st = isvd_set_tuning(op, &cands[i], stream);
      if (st != ISVD_OK) break;
      st = isvd_apply(op, G, ld, b, Y, ld, dtype, stream);  // warm-up (and workspace growth)
      if (st != ISVD_OK) break;
      float ms = 0.f;
      for (int rep = 0; rep < 3 && st == ISVD_OK; ++rep) {
        cudaEventRecord(e0, s);
        st = isvd_apply(op, G, ld, b, Y, ld, dtype, stream);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(ISVD_ERR_CUDA, "timing failed");
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        ms = rep == 0 ? t : (t < ms ? t : ms);
      }
      if (st == ISVD_OK && ms < best_ms) {
        best_ms = ms;
        best = cands[i];
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  if (G) op_free(op, G, s);
  if (Y) op_free(op, Y, s);
  if (st != ISVD_OK) {
    const std::string keep = isvd::last_error();
    isvd_set_tuning(op, &base, stream);
    isvd::set_error("%s", keep.c_str());
    return st;
  }
  ISVD_TRY(isvd_set_tuning(op, &best, stream));
  if (cache_path) cache_store(cache_path, key, best);
  if (out) *out = best;
  return ISVD_OK;
}

}  // extern "C"
