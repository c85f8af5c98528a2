// Alg. 1 (App. A.2): randomized range finder with power iterations,
// CholeskyQR orthonormalisation (Alg. 2, right) and Rayleigh-Ritz, as one
// stream-ordered sequence that is captured once into a CUDA graph.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <set>
#include <vector>

#include "internal.h"

namespace isvd {

// CholeskyQR2 with conditional extra passes after a shifted one (passes 3, 4
// return at once unless a shift happened in the two passes before them).
isvd_status orth_enqueue(void *Q, int64_t ldq, int dt, int64_t rows, int32_t l, double *Racc, const OrthBufs &o,
                         isvd_info *info, cudaStream_t s) {
  ISVD_CUDA_TRY(orth_reset_launch(o.state, s));
  if (Racc) ISVD_CUDA_TRY(racc_init_launch(Racc, l, s));
  for (int pass = 1; pass <= 4; ++pass) {
    PassGate g{o.state, pass};
    ISVD_CUDA_TRY(gram_launch(Q, ldq, dt, rows, l, o.gram_partial, o.n_part, o.W, g, s));
    ISVD_CUDA_TRY(chol_inv_launch(o.W, l, rows, dt, o.Rinv, l, nullptr, Racc, o.tmp, o.state, info, pass, s));
    ISVD_CUDA_TRY(gemm_tri_inplace_launch(Q, ldq, dt, rows, l, o.Rinv, l, g, s, o.colsum));
  }
  return ISVD_OK;
}

namespace {

__global__ void cast_kernel_bf16_f32(const __nv_bfloat16 *in, float *out, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = __bfloat162float(in[i]);
}

struct Carver {
  char *base;
  size_t off = 0;
  template <typename T>
  T *take(size_t count) {
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += (size_t)round_up((int64_t)(sizeof(T) * count), 256);
    return p;
  }
};

// OrthBufs for blocks of width l; above ISVD_MAX_BLOCK the CholeskyQR2
// buffers serve the 128-column panels of the wide path, which adds its own
// (`wide`, may be null when l <= ISVD_MAX_BLOCK).
void carve_orth(Carver &c, int64_t rows, int32_t l, OrthBufs *o, char **wide = nullptr, bool colsum = false) {
  if (l > ISVD_MAX_BLOCK) {
    char *w = c.take<char>(wide_orth_bytes(rows, l));
    if (wide) *wide = w;
    l = ISVD_MAX_BLOCK;
  }
  o->n_part = gram_partials(rows);
  o->gram_partial = c.take<double>((size_t)o->n_part * l * l);
  o->W = c.take<double>((size_t)l * l);
  o->tmp = c.take<double>((size_t)l * l);
  o->Rinv = c.take<float>((size_t)l * l);
  o->state = c.take<int32_t>(kOrthStateInts);
  o->colsum = colsum ? c.take<double>((size_t)gemm_colsum_parts(rows) * l) : nullptr;
}

// Q (rows x l) <- its orthonormal factor: one CholeskyQR2 up to
// ISVD_MAX_BLOCK columns, 128-column panels (FP32) above
isvd_status orth_any(void *Q, int64_t ldq, int dt, int64_t rows, int32_t l, double *Racc, const OrthBufs &o,
                     char *wide, isvd_info *info, cudaStream_t s) {
  if (l <= ISVD_MAX_BLOCK) return orth_enqueue(Q, ldq, dt, rows, l, Racc, o, info, s);
  if (dt != DT_F32 || !wide) return fail(ISVD_ERR_UNSUPPORTED, "blocks wider than %d are FP32 only", ISVD_MAX_BLOCK);
  return wide_orth_enqueue((float *)Q, ldq, rows, l, Racc, o, wide, info, s);
}

struct SvdPlan {
  int32_t k, p, l, ld, iters;
  uint64_t seed;
  int prec;
  float *U, *S, *V;
  int64_t ldu, ldv;
  isvd_info *info;
};

struct SvdBufs {
  void *qr, *qc;        // blocks in the iteration dtype
  float *qr32, *qc32;   // FP32 blocks (alias qr/qc in FP32 mode)
  char *apply_base;
  OrthBufs orth;
  char *wide = nullptr;  // panel buffers of blocks wider than ISVD_MAX_BLOCK
  double *Racc, *Uo, *So, *Vo, *jwork;
  float *Lk, *Rk;
  isvd_info *info;
};

size_t carve_svd(const isvd_operator *op, const SvdPlan &P, char *base, SvdBufs *b) {
  Carver c{base};
  const int64_t rows = op->rows, cols = op->cols;
  const bool mixed = P.prec == ISVD_PREC_MIXED;
  const size_t es = mixed ? 2 : 4;
  b->qr = c.take<char>(es * rows * P.ld);
  b->qc = c.take<char>(es * cols * P.ld);
  if (mixed) {
    b->qr32 = c.take<float>((size_t)rows * P.ld);
    b->qc32 = c.take<float>((size_t)cols * P.ld);
  } else {
    b->qr32 = (float *)b->qr;
    b->qc32 = (float *)b->qc;
  }
  const size_t ab = std::max(apply_scratch_bytes(op, P.l, DT_F32, false), apply_scratch_bytes(op, P.l, DT_F32, true));
  b->apply_base = c.take<char>(ab);
  // the Q R^-1 passes also form the column sums of their result when the
  // operator's next product wants 1^T Q (the all-ones term of a leaf)
  const isvd_operator_desc &d = op->desc;
  const bool colsum = P.l <= ISVD_MAX_BLOCK && op->compose < 0 && d.form == ISVD_FORM_POLY && d.ones_coeff != 0.0 &&
                      d.lr_rank == 0 && !d.gather_rows && op->rows == op->cols;
  carve_orth(c, std::max(rows, cols), P.l, &b->orth, &b->wide, colsum);
  b->Racc = c.take<double>((size_t)P.l * P.l);
  b->Uo = c.take<double>((size_t)P.l * P.l);
  b->Vo = c.take<double>((size_t)P.l * P.l);
  b->So = c.take<double>((size_t)P.l);
  b->jwork = c.take<double>(small_svd_work_doubles(P.l));
  b->Lk = c.take<float>((size_t)P.l * P.k);
  b->Rk = c.take<float>((size_t)P.l * P.k);
  b->info = c.take<isvd_info>(1);
  return c.off;
}

// `fresh`: `in` is the block the last orthonormalisation wrote, whose column
// sums that step formed
isvd_status apply_step(isvd_operator *op, const void *in, void *out, int32_t l, int64_t ld, int dt, bool transpose,
                       const SvdBufs &b, cudaStream_t s, bool fresh = false) {
  ApplyScratch sc;
  apply_scratch_carve(op, l, dt, transpose, b.apply_base, &sc);
  if (fresh && b.orth.colsum) {
    sc.ones_parts = b.orth.colsum;
    sc.ones_nparts = gemm_colsum_parts(op->rows);  // rows == cols when colsum is carved
    sc.ones_ld = l;
  }
  return apply_impl(op, in, ld, l, out, ld, dt, transpose, sc, s);
}

isvd_status svd_enqueue(isvd_operator *op, const SvdPlan &P, const SvdBufs &b, cudaStream_t s) {
  const int64_t rows = op->rows, cols = op->cols;
  const bool mixed = P.prec == ISVD_PREC_MIXED;
  const int dt = mixed ? DT_BF16 : DT_F32;
  isvd_info *info = P.info ? P.info : b.info;
  ISVD_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(isvd_info), s));
  // Q ~ N(0,1)^{c x l}
  ISVD_CUDA_TRY(gaussian_launch(P.seed, cols, P.l, b.qc, P.ld, dt, s));
  for (int it = 0; it < P.iters; ++it) {
    ISVD_TRY(apply_step(op, b.qc, b.qr, P.l, P.ld, dt, false, b, s, it > 0));  // M Q
    ISVD_TRY(orth_any(b.qr, P.ld, dt, rows, P.l, nullptr, b.orth, b.wide, info, s));
    ISVD_TRY(apply_step(op, b.qr, b.qc, P.l, P.ld, dt, true, b, s, true));     // M^T Q
    ISVD_TRY(orth_any(b.qc, P.ld, dt, cols, P.l, nullptr, b.orth, b.wide, info, s));
  }
  if (mixed) {
    // the refinement step and the Rayleigh-Ritz step run in FP32
    const int64_t n = cols * P.ld;
    int64_t blocks = std::min<int64_t>(ceil_div(n, 256), kNumSMs * 16);
    cast_kernel_bf16_f32<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>((const __nv_bfloat16 *)b.qc,
                                                                                 b.qc32, n);
    ISVD_CUDA_TRY(cudaGetLastError());
  }
  // (in mixed precision qc32 holds qc's values exactly: its column sums stand)
  ISVD_TRY(apply_step(op, b.qc32, b.qr32, P.l, P.ld, DT_F32, false, b, s, P.iters > 0));
  ISVD_TRY(orth_any(b.qr32, P.ld, DT_F32, rows, P.l, nullptr, b.orth, b.wide, info, s));
  // B^T = M^T Q = Qt R  (CholeskyQR of B^T, R accumulated over the passes)
  ISVD_TRY(apply_step(op, b.qr32, b.qc32, P.l, P.ld, DT_F32, true, b, s, true));
  ISVD_TRY(orth_any(b.qc32, P.ld, DT_F32, cols, P.l, b.Racc, b.orth, b.wide, info, s));
  // B = R^T Qt^T;  R = Uo S Vo^T  =>  B = Vo S (Qt Uo)^T:  U = Q Vo, V = Qt Uo
  ISVD_CUDA_TRY(small_svd_launch(b.Racc, P.l, b.Uo, b.So, b.Vo, b.jwork, /*Uk=*/b.Rk, /*Vk=*/b.Lk, /*Sk=*/P.S, P.k,
                                 info, P.iters, s));
  // U = Q Vo_k, V = Qt Uo_k: tensor cores where the layout allows, else CUDA cores
  auto product = [&](const float *Qb, int64_t n, const float *Bk, float *Out, int64_t ldo) -> cudaError_t {
    bool launched = false;
    cudaError_t e = gemm_tc_launch(Qb, P.ld, n, P.l, Bk, P.k, P.k, Out, ldo, &launched, s);
    if (e == cudaSuccess && !launched)
      e = gemm_small_launch(Qb, P.ld, DT_F32, n, P.l, Bk, P.k, P.k, false, Out, ldo, DT_F32, PassGate{}, s);
    return e;
  };
  ISVD_CUDA_TRY(product(b.qr32, rows, b.Lk, P.U, P.ldu));
  ISVD_CUDA_TRY(product(b.qc32, cols, b.Rk, P.V, P.ldv));
  return ISVD_OK;
}

int64_t count_kernel_nodes(cudaGraph_t graph) {
  int64_t kernels = 0;
  size_t nn = 0;
  if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn > 0) {
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
      for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
      }
  }
  return kernels;
}

// ---- many independent problems in one graph ----------------------------------
// The problems are spread over kBatchBranches parallel branches of one graph
// (longest first onto the least-loaded branch), so that small problems,
// whose kernels fill a fraction of the GPU each, run side by side.
constexpr int kBatchBranches = 16;
constexpr size_t kMaxBatchedGraphs = 4;

struct BatchedGraph {
  std::vector<uint64_t> key;
  std::vector<uint64_t> serials;
  cudaGraphExec_t exec = nullptr;
  int64_t kernel_nodes = 0;
};
std::mutex g_batched_mu;
std::vector<BatchedGraph> g_batched;
thread_local int64_t t_batched_kernel_nodes = -1;

// Side streams and events of one fork/join; released after the capture ends.
struct Fork {
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  ~Fork() {
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    for (cudaStream_t t : streams) cudaStreamDestroy(t);
  }
};

double problem_cost(const isvd_operator *op, const SvdPlan &P) {
  const double nnz = (double)op->desc.A.nnz + (double)op->x_nnz;
  const double deg = op->desc.form == ISVD_FORM_POLY ? std::max(1, op->desc.degree) : op->desc.L + 1;
  const double dim = (double)(op->rows + op->cols);
  return (2.0 * P.iters + 2.0) * ((nnz * deg + dim) * P.l + dim * (double)P.l * P.l);
}

isvd_status batched_enqueue(isvd_operator *const *ops, const std::vector<SvdPlan> &plans,
                            const std::vector<SvdBufs> &bufs, Fork &fork, cudaStream_t s) {
  const int count = (int)plans.size();
  const int B = std::min(count, kBatchBranches);
  std::vector<int> order(count);
  std::vector<double> cost(count);
  for (int i = 0; i < count; ++i) {
    order[i] = i;
    cost[i] = problem_cost(ops[i], plans[i]);
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<std::vector<int>> lanes(B);
  std::vector<double> load(B, 0.0);
  for (int i : order) {
    const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lanes[b].push_back(i);
    load[b] += cost[i];
  }
  fork.streams.assign(B, nullptr);
  fork.events.assign(B + 1, nullptr);
  for (int b = 0; b <= B; ++b) ISVD_CUDA_TRY(cudaEventCreateWithFlags(&fork.events[b], cudaEventDisableTiming));
  for (int b = 0; b < B; ++b) ISVD_CUDA_TRY(cudaStreamCreateWithFlags(&fork.streams[b], cudaStreamNonBlocking));
  ISVD_CUDA_TRY(cudaEventRecord(fork.events[B], s));
  isvd_status first = ISVD_OK;
  for (int b = 0; b < B; ++b) {
    ISVD_CUDA_TRY(cudaStreamWaitEvent(fork.streams[b], fork.events[B], 0));
    for (int i : lanes[b]) {
      if (first != ISVD_OK) break;
      first = svd_enqueue(ops[i], plans[i], bufs[i], fork.streams[b]);
    }
    // join every branch, also after a failure, so that a capture can end
    ISVD_CUDA_TRY(cudaEventRecord(fork.events[b], fork.streams[b]));
    ISVD_CUDA_TRY(cudaStreamWaitEvent(s, fork.events[b], 0));
  }
  return first;
}

}  // namespace

void batched_forget(uint64_t serial) {
  std::lock_guard<std::mutex> lk(g_batched_mu);
  for (size_t i = 0; i < g_batched.size();) {
    BatchedGraph &e = g_batched[i];
    if (std::find(e.serials.begin(), e.serials.end(), serial) != e.serials.end()) {
      cudaGraphExecDestroy(e.exec);
      g_batched.erase(g_batched.begin() + (std::ptrdiff_t)i);
    } else {
      ++i;
    }
  }
}

}  // namespace isvd

using namespace isvd;

extern "C" {

isvd_status isvd_svd(isvd_operator *op, int32_t k, int32_t oversample, int32_t iters, uint64_t seed,
                     isvd_precision precision, float *U, int64_t ldu, float *S, float *V, int64_t ldv,
                     isvd_info *dev_info, void *stream) {
  if (!op || !U || !S || !V) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  if (k < 1 || oversample < 0 || iters < 0) return fail(ISVD_ERR_INVALID_ARGUMENT, "need k >= 1, oversample >= 0, iters >= 0");
  if (precision != ISVD_PREC_FP32 && precision != ISVD_PREC_MIXED)
    return fail(ISVD_ERR_INVALID_ARGUMENT, "unknown precision");
  const int64_t l = (int64_t)k + oversample;
  if (l > ISVD_MAX_BLOCK_WIDE)
    return fail(ISVD_ERR_UNSUPPORTED, "block width k + oversample = %lld > %d", (long long)l, ISVD_MAX_BLOCK_WIDE);
  if (l > ISVD_MAX_BLOCK && precision != ISVD_PREC_FP32)
    return fail(ISVD_ERR_UNSUPPORTED, "block widths above %d run in FP32 only", ISVD_MAX_BLOCK);
  if (l > std::min(op->rows, op->cols))
    return fail(ISVD_ERR_SHAPE, "block width k + oversample = %lld exceeds min(rows, cols)", (long long)l);
  if (ldu < k || ldv < k) return fail(ISVD_ERR_INVALID_ARGUMENT, "ldu and ldv must be >= k");
  cudaStream_t s = (cudaStream_t)stream;
  SvdPlan P{};
  P.k = k;
  P.p = oversample;
  P.l = (int32_t)l;
  P.ld = (int32_t)round_up(l, 8);
  P.iters = iters;
  P.seed = seed;
  P.prec = precision;
  P.U = U;
  P.S = S;
  P.V = V;
  P.ldu = ldu;
  P.ldv = ldv;
  P.info = dev_info;
  SvdBufs b{};
  const size_t bytes = carve_svd(op, P, nullptr, &b);
  ISVD_TRY(ensure_arena(op, bytes, s));
  carve_svd(op, P, (char *)op->arena, &b);

  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  ISVD_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) return svd_enqueue(op, P, b, s);  // caller is capturing

  uint64_t key[16] = {(uint64_t)k,      (uint64_t)oversample, (uint64_t)iters,     seed,
                      (uint64_t)precision, (uint64_t)(uintptr_t)U, (uint64_t)ldu, (uint64_t)(uintptr_t)S,
                      (uint64_t)(uintptr_t)V, (uint64_t)ldv, (uint64_t)(uintptr_t)dev_info,
                      (uint64_t)(uintptr_t)op->arena, tree_generation(op), 0, 0, 0};
  for (auto &g : op->graphs) {
    if (memcmp(g.key, key, sizeof key) == 0) {
      op->last_kernel_nodes = g.kernel_nodes;
      ISVD_CUDA_TRY(cudaGraphLaunch(g.exec, s));
      return ISVD_OK;
    }
  }
  cudaGraph_t graph = nullptr;
  ISVD_CUDA_TRY(cudaStreamBeginCapture(op->capture_stream, cudaStreamCaptureModeThreadLocal));
  const isvd_status st = svd_enqueue(op, P, b, op->capture_stream);
  const cudaError_t ce = cudaStreamEndCapture(op->capture_stream, &graph);
  if (st != ISVD_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(ISVD_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
  }
  const int64_t kernels = count_kernel_nodes(graph);
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return fail(ISVD_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ie));
  if (op->graphs.size() >= 8) {
    cudaGraphExecDestroy(op->graphs.front().exec);
    op->graphs.erase(op->graphs.begin());
  }
  isvd_operator::GraphEntry e;
  memcpy(e.key, key, sizeof key);
  e.exec = exec;
  e.kernel_nodes = kernels;
  op->graphs.push_back(e);
  op->last_kernel_nodes = kernels;
  ISVD_CUDA_TRY(cudaGraphLaunch(exec, s));
  return ISVD_OK;
}

int64_t isvd_graph_kernel_nodes(const isvd_operator *op) { return op ? op->last_kernel_nodes : -1; }

isvd_status isvd_svd_batched(isvd_operator *const *ops, const int32_t *k, int32_t count, int32_t oversample,
                             int32_t iters, uint64_t seed, isvd_precision precision, float *const *U,
                             float *const *S, float *const *V, isvd_info *dev_info, void *stream) {
  if (!ops || !k || !U || !S || !V || count < 1) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument or count < 1");
  if (oversample < 0 || iters < 0) return fail(ISVD_ERR_INVALID_ARGUMENT, "need oversample >= 0, iters >= 0");
  if (precision != ISVD_PREC_FP32 && precision != ISVD_PREC_MIXED)
    return fail(ISVD_ERR_INVALID_ARGUMENT, "unknown precision");
  cudaStream_t s = (cudaStream_t)stream;
  std::set<const isvd_operator *> seen;
  std::vector<SvdPlan> plans(count);
  std::vector<SvdBufs> bufs(count);
  std::vector<uint64_t> key = {(uint64_t)count, (uint64_t)oversample, (uint64_t)iters, seed, (uint64_t)precision,
                               (uint64_t)(uintptr_t)dev_info};
  std::vector<uint64_t> serials(count);
  for (int i = 0; i < count; ++i) {
    isvd_operator *op = ops[i];
    if (!op || !U[i] || !S[i] || !V[i]) return fail(ISVD_ERR_INVALID_ARGUMENT, "null pointer for problem %d", i);
    if (op->compose >= 0)
      return fail(ISVD_ERR_UNSUPPORTED, "problem %d: composite operators are not batched (children may be shared)", i);
    if (!seen.insert(op).second)
      return fail(ISVD_ERR_INVALID_ARGUMENT, "problem %d repeats an operator (each needs its own workspace)", i);
    const int64_t l = (int64_t)k[i] + oversample;
    if (k[i] < 1) return fail(ISVD_ERR_INVALID_ARGUMENT, "problem %d: k < 1", i);
    if (l > ISVD_MAX_BLOCK) return fail(ISVD_ERR_UNSUPPORTED, "problem %d: k + oversample > %d", i, ISVD_MAX_BLOCK);
    if (l > std::min(op->rows, op->cols))
      return fail(ISVD_ERR_SHAPE, "problem %d: k + oversample exceeds min(rows, cols)", i);
    SvdPlan &P = plans[i];
    P.k = k[i];
    P.p = oversample;
    P.l = (int32_t)l;
    P.ld = (int32_t)round_up(l, 8);
    P.iters = iters;
    P.seed = seed + (uint64_t)i;
    P.prec = precision;
    P.U = U[i];
    P.S = S[i];
    P.V = V[i];
    P.ldu = k[i];
    P.ldv = k[i];
    P.info = dev_info ? dev_info + i : nullptr;
    const size_t bytes = carve_svd(op, P, nullptr, &bufs[i]);
    ISVD_TRY(ensure_arena(op, bytes, s));
    carve_svd(op, P, (char *)op->arena, &bufs[i]);
  }
  for (int i = 0; i < count; ++i) {
    const isvd_operator *op = ops[i];
    serials[i] = op->serial;
    const uint64_t e[7] = {op->serial, op->generation, (uint64_t)k[i], (uint64_t)(uintptr_t)U[i],
                           (uint64_t)(uintptr_t)S[i], (uint64_t)(uintptr_t)V[i], (uint64_t)(uintptr_t)op->arena};
    key.insert(key.end(), e, e + 7);
  }

  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  ISVD_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) {  // the caller is capturing: fork inside its graph
    Fork fork;
    return batched_enqueue(ops, plans, bufs, fork, s);
  }
  {
    std::lock_guard<std::mutex> lk(g_batched_mu);
    for (BatchedGraph &g : g_batched)
      if (g.key == key) {
        t_batched_kernel_nodes = g.kernel_nodes;
        ISVD_CUDA_TRY(cudaGraphLaunch(g.exec, s));
        return ISVD_OK;
      }
  }
  cudaStream_t cs = ops[0]->capture_stream;
  cudaGraph_t graph = nullptr;
  isvd_status st;
  cudaError_t ce;
  {
    Fork fork;
    ISVD_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    st = batched_enqueue(ops, plans, bufs, fork, cs);
    ce = cudaStreamEndCapture(cs, &graph);
  }
  if (st != ISVD_OK || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (st != ISVD_OK) return st;
    return fail(ISVD_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
  }
  BatchedGraph e;
  e.key = key;
  e.serials = serials;
  e.kernel_nodes = count_kernel_nodes(graph);
  const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return fail(ISVD_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ie));
  t_batched_kernel_nodes = e.kernel_nodes;
  ISVD_CUDA_TRY(cudaGraphLaunch(e.exec, s));
  std::lock_guard<std::mutex> lk(g_batched_mu);
  if (g_batched.size() >= kMaxBatchedGraphs) {
    cudaGraphExecDestroy(g_batched.front().exec);
    g_batched.erase(g_batched.begin());
  }
  g_batched.push_back(std::move(e));
  return ISVD_OK;
}

int64_t isvd_batched_kernel_nodes(void) { return t_batched_kernel_nodes; }



isvd_status isvd_gaussian(uint64_t seed, int64_t rows, int32_t cols, void *out, int64_t ld, isvd_dtype dtype,
                          void *stream) {
  if (!out || rows < 0 || cols < 0 || ld < cols || ld % 8) return fail(ISVD_ERR_INVALID_ARGUMENT, "bad block arguments");
  if (dtype != ISVD_F32 && dtype != ISVD_BF16) return fail(ISVD_ERR_INVALID_ARGUMENT, "unknown dtype");
  ISVD_CUDA_TRY(gaussian_launch(seed, rows, cols, out, ld, dtype == ISVD_F32 ? DT_F32 : DT_BF16, (cudaStream_t)stream));
  return ISVD_OK;
}

isvd_status isvd_philox_words(uint64_t seed, int64_t rows, uint32_t *out, void *stream) {
  if (!out || rows < 0) return fail(ISVD_ERR_INVALID_ARGUMENT, "bad arguments");
  ISVD_CUDA_TRY(philox_words_launch(seed, rows, out, (cudaStream_t)stream));
  return ISVD_OK;
}

isvd_status isvd_orthonormalize(isvd_operator *op, float *Q, int64_t rows, int32_t l, int64_t ldq, double *R_out,
                                isvd_info *dev_info, void *stream) {
  if (!op || !Q) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  if (l < 1 || l > ISVD_MAX_BLOCK_WIDE || rows < l)
    return fail(ISVD_ERR_SHAPE, "need 1 <= l <= min(rows, %d)", ISVD_MAX_BLOCK_WIDE);
  if (ldq < l || ldq % 8 || (uintptr_t)Q % 16)
    return fail(ISVD_ERR_INVALID_ARGUMENT, "ldq must be >= l and a multiple of 8, Q 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  Carver c{nullptr};
  OrthBufs o;
  char *wide = nullptr;
  carve_orth(c, rows, l, &o, &wide);
  c.take<isvd_info>(1);
  ISVD_TRY(ensure_arena(op, c.off, s));
  Carver c2{(char *)op->arena};
  carve_orth(c2, rows, l, &o, &wide);
  isvd_info *own = c2.take<isvd_info>(1);
  isvd_info *info = dev_info ? dev_info : own;
  if (!dev_info) ISVD_CUDA_TRY(cudaMemsetAsync(own, 0, sizeof(isvd_info), s));
  return orth_any(Q, ldq, DT_F32, rows, l, R_out, o, wide, info, s);
}

isvd_status isvd_closed_form(isvd_operator *op, const float *U, int64_t ldu, const float *S, const float *V,
                             int64_t ldv, int32_t k, const float *Y, int64_t ldy, int32_t m, double rcond, float *W,
                             int64_t ldw, void *stream) {
  if (!op || !U || !S || !V || !Y || !W) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  if (k < 1 || k > ISVD_MAX_BLOCK || m < 1 || m > ISVD_MAX_BLOCK)
    return fail(ISVD_ERR_SHAPE, "need 1 <= k, m <= %d", ISVD_MAX_BLOCK);
  if (k > std::min(op->rows, op->cols)) return fail(ISVD_ERR_SHAPE, "k exceeds min(rows, cols)");
  if (ldu < k || ldv < k || ldy < m || ldw < m) return fail(ISVD_ERR_INVALID_ARGUMENT, "leading dimension too small");
  if (!(rcond >= 0.0)) return fail(ISVD_ERR_INVALID_ARGUMENT, "rcond must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const int32_t parts = closed_form_parts(op->rows, k, m);
  Carver c{nullptr};
  c.take<double>((size_t)parts * k * m);
  c.take<float>((size_t)k * m);
  ISVD_TRY(ensure_arena(op, c.off, s));
  Carver c2{(char *)op->arena};
  double *partial = c2.take<double>((size_t)parts * k * m);
  float *Z = c2.take<float>((size_t)k * m);
  ISVD_CUDA_TRY(closed_form_launch(U, ldu, S, V, ldv, op->rows, op->cols, k, Y, ldy, m, rcond, W, ldw, partial, parts,
                                   Z, s));
  return ISVD_OK;
}

isvd_status isvd_embed(const float *X, int64_t ldx, int64_t rows, int32_t k, const float *S, float *out,
                       int64_t ldo, void *stream) {
  if (!X || !S || !out) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  if (k < 1) return fail(ISVD_ERR_SHAPE, "need k >= 1");
  if (rows < 0) return fail(ISVD_ERR_INVALID_ARGUMENT, "rows must be >= 0");
  if (ldx < k || ldo < k) return fail(ISVD_ERR_INVALID_ARGUMENT, "leading dimension too small");
  ISVD_CUDA_TRY(embed_launch(X, ldx, rows, k, S, out, ldo, (cudaStream_t)stream));
  return ISVD_OK;
}

isvd_status isvd_pair_scores(const float *L, int64_t ldl, int64_t rows, const float *R, int64_t ldr, int64_t cols,
                             int32_t k, const int32_t *src, const int32_t *dst, int64_t n_pairs, float *out,
                             isvd_info *dev_info, void *stream) {
  if (n_pairs < 0) return fail(ISVD_ERR_INVALID_ARGUMENT, "n_pairs must be >= 0");
  if (n_pairs == 0) return ISVD_OK;
  if (!L || !R || !src || !dst || !out) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  if (k < 1) return fail(ISVD_ERR_SHAPE, "need k >= 1");
  if (rows < 0 || cols < 0) return fail(ISVD_ERR_INVALID_ARGUMENT, "rows and cols must be >= 0");
  if (ldl < k || ldr < k) return fail(ISVD_ERR_INVALID_ARGUMENT, "leading dimension too small");
  ISVD_CUDA_TRY(pair_scores_launch(L, ldl, rows, R, ldr, cols, k, src, dst, n_pairs, out, dev_info,
                                   (cudaStream_t)stream));
  return ISVD_OK;
}

isvd_status isvd_small_svd(isvd_operator *op, const double *A, int32_t l, double *Uo, double *S, double *Vo,
                           isvd_info *dev_info, void *stream) {
  if (!op || !A || !Uo || !S || !Vo) return fail(ISVD_ERR_INVALID_ARGUMENT, "null argument");
  if (l < 1 || l > ISVD_MAX_BLOCK_WIDE) return fail(ISVD_ERR_SHAPE, "need 1 <= l <= %d", ISVD_MAX_BLOCK_WIDE);
  cudaStream_t s = (cudaStream_t)stream;
  Carver c{nullptr};
  c.take<double>(small_svd_work_doubles(l));
  ISVD_TRY(ensure_arena(op, c.off, s));
  // iters = -1: dev_info->iters_done receives the Jacobi sweep count
  ISVD_CUDA_TRY(small_svd_launch(A, l, Uo, S, Vo, (double *)op->arena, nullptr, nullptr, nullptr, 0, dev_info, -1, s));
  return ISVD_OK;
}

}  // extern "C"
