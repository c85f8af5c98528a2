// Allocation-free CholeskyQR2 entry point.
//
// Some callers cannot allocate device memory at the point where they need an
// orthonormalisation: code running inside another framework's allocator or
// memory-pool callback (where re-entering the allocator would deadlock or
// corrupt its state), and latency-bound services that reserve all device
// memory up front and forbid cudaMalloc on the hot path because it can
// synchronise the device.  isvd_orthonormalize_noalloc serves them: its
// scratch (Gram partials, the l x l matrices and the pass state) lives in one
// file-scope __device__ array of fixed size, so the call allocates nothing.
#include <mutex>

#include "internal.h"

namespace isvd {
namespace {

constexpr int32_t kNoallocMaxBlock = ISVD_NOALLOC_MAX_BLOCK;
constexpr int32_t kNoallocMaxPartials = 2 * kNumSMs;  // the largest Gram partial count

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kPartialBytes = align256(sizeof(double) * kNoallocMaxPartials * kNoallocMaxBlock * kNoallocMaxBlock);
constexpr size_t kSquareF64 = align256(sizeof(double) * kNoallocMaxBlock * kNoallocMaxBlock);
constexpr size_t kSquareF32 = align256(sizeof(float) * kNoallocMaxBlock * kNoallocMaxBlock);
constexpr size_t kStateBytes = align256(sizeof(int32_t) * kOrthStateInts);
constexpr size_t kInfoBytes = align256(sizeof(isvd_info));
constexpr size_t kScratchBytes = kPartialBytes + 2 * kSquareF64 + kSquareF32 + kStateBytes + kInfoBytes;

// Shared by every call on a device; kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// Once per device, with that device current: the device address of the array
// (in host code its name is only a host-side stand-in).  The kernel
// attributes the orthonormalisation kernels need are set here too, but once
// per process (the library's init functions), so the library serves one
// device per process.
isvd_status setup_device(unsigned char **out) {
  int dev = 0;
  ISVD_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(ISVD_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    ISVD_CUDA_TRY(small_kernels_init());
    ISVD_CUDA_TRY(dense_kernels_init());
    void *p = nullptr;
    ISVD_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_scratch_addr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_addr[dev];
  return ISVD_OK;
}

}  // namespace
}  // namespace isvd

using namespace isvd;

extern "C" isvd_status isvd_orthonormalize_noalloc(float *Q, int64_t rows, int32_t l, int64_t ldq, double *R_out,
                                                   isvd_info *dev_info, void *stream) {
  if (!Q) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  if (l < 1 || l > kNoallocMaxBlock)
    return fail(ISVD_ERR_UNSUPPORTED, "isvd_orthonormalize_noalloc: block width %d outside 1..%d (fixed scratch size)",
                l, kNoallocMaxBlock);
  if (rows < l) return fail(ISVD_ERR_SHAPE, "need rows >= l");
  if (ldq < l || ldq % 8 || (uintptr_t)Q % 16)
    return fail(ISVD_ERR_INVALID_ARGUMENT, "ldq must be >= l and a multiple of 8, Q 16-byte aligned");
  unsigned char *base = nullptr;
  ISVD_TRY(setup_device(&base));
  OrthBufs o;
  o.n_part = gram_partials(rows);  // at most kNoallocMaxPartials
  size_t off = 0;
  o.gram_partial = reinterpret_cast<double *>(base + off);
  off += kPartialBytes;
  o.W = reinterpret_cast<double *>(base + off);
  off += kSquareF64;
  o.tmp = reinterpret_cast<double *>(base + off);
  off += kSquareF64;
  o.Rinv = reinterpret_cast<float *>(base + off);
  off += kSquareF32;
  o.state = reinterpret_cast<int32_t *>(base + off);  // reset by the first kernel of every call
  off += kStateBytes;
  isvd_info *own_info = reinterpret_cast<isvd_info *>(base + off);
  cudaStream_t s = (cudaStream_t)stream;
  isvd_info *info = dev_info;
  if (!info) {
    // the array keeps the previous call's status: clear it
    ISVD_CUDA_TRY(cudaMemsetAsync(own_info, 0, sizeof(isvd_info), s));
    info = own_info;
  }
  return orth_enqueue(Q, ldq, DT_F32, rows, l, R_out, o, info, s);
}
