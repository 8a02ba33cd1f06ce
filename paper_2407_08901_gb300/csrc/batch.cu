// Many independent eigenproblems solved together (batched workload: dozens of
// Hamiltonians of uneven sizes).  One problem of a few ten thousand rows leaves
// most of the GPU idle (short kernels, host round trips between steps), so a
// pool of host threads, each driving its own non-blocking CUDA stream, keeps
// several solves in flight.  Problems are taken from a shared counter in
// decreasing order of stored entries (longest first), which bounds the tail.
// Each solve is the ordinary sppc_solve on its own handle: results are
// identical to solving the problems one after another.
#include <algorithm>
#include <atomic>
#include <numeric>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "sppc.h"
#include "sppc_internal.h"

namespace sppc {
void handle_size(sppc_handle h, int64_t* n, int64_t* nnz, int* k);
sppc_status handle_fail(sppc_handle h, sppc_status st, const char* msg);
}  // namespace sppc

extern "C" sppc_status sppc_solve_batch(sppc_handle* handles, int32_t count, double tol, int32_t workers,
                                        int32_t kmax, double* theta, double* resid, int32_t* converged,
                                        sppc_stats* stats) {
  using namespace sppc;
  if (!handles || count < 1 || workers < 1 || kmax < 1 || !theta || !resid || !converged)
    return handle_fail(nullptr, SPPC_ERR_ARG, "sppc_solve_batch: bad arguments");
  std::vector<int64_t> nnz(count);
  for (int32_t i = 0; i < count; ++i) {
    if (!handles[i]) return handle_fail(nullptr, SPPC_ERR_ARG, "sppc_solve_batch: NULL handle");
    int k = 0;
    handle_size(handles[i], nullptr, &nnz[i], &k);
    if (k > kmax) return handle_fail(nullptr, SPPC_ERR_ARG, "sppc_solve_batch: a handle has k > kmax");
  }
  std::vector<int32_t> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return nnz[a] > nnz[b]; });
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return handle_fail(nullptr, SPPC_ERR_CUDA, "sppc_solve_batch: no device");
  std::fill(theta, theta + (size_t)count * kmax, 0.0);
  std::fill(resid, resid + (size_t)count * kmax, 0.0);
  std::vector<sppc_status> status(count, SPPC_OK);
  std::atomic<int32_t> next{0};
  std::atomic<int> setup_error{0};
  auto work = [&] {
    cudaStream_t s = nullptr;
    if (cudaSetDevice(dev) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      setup_error.store(1);
      return;
    }
    for (;;) {
      const int32_t t = next.fetch_add(1);
      if (t >= count) break;
      const int32_t i = order[t];
      sppc_stats st{};
      status[i] = sppc_solve(handles[i], tol, -1, theta + (size_t)i * kmax, nullptr, 0, resid + (size_t)i * kmax, &st, s);
      converged[i] = status[i] == SPPC_OK ? 1 : 0;
      if (stats) stats[i] = st;
    }
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  };
  const int nw = std::min<int32_t>(workers, count);
  std::vector<std::thread> pool;
  pool.reserve(nw);
  for (int w = 0; w < nw; ++w) pool.emplace_back(work);
  for (auto& th : pool) th.join();
  if (setup_error.load()) return handle_fail(nullptr, SPPC_ERR_CUDA, "sppc_solve_batch: stream setup failed");
  // first hard error (by problem index), else NOT_CONVERGED if any missed tol
  for (int32_t i = 0; i < count; ++i)
    if (status[i] != SPPC_OK && status[i] != SPPC_NOT_CONVERGED) return status[i];
  for (int32_t i = 0; i < count; ++i)
    if (status[i] == SPPC_NOT_CONVERGED) return SPPC_NOT_CONVERGED;
  return SPPC_OK;
}

// ---------------------------------------------------------------- batched SpMM
// A plan: the products Y_i = H_i X_i of `count` handles in one persistent launch
// (k_spmm_batch.cu), with the FP64 <-> double-float conversions around it, all
// captured once in a CUDA graph and replayed by sppc_spmm_batch_run.
struct sppc_batch_plan_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  sppc::BatchItem* items = nullptr;
  int64_t* prefix = nullptr;
  unsigned long long* queue = nullptr;
};

namespace sppc {
const SellDev* handle_matrix(sppc_handle h, int64_t* n);
void handle_scratch(sppc_handle h, float2** t1, float2** t2);
}  // namespace sppc

extern "C" sppc_status sppc_spmm_batch_destroy(sppc_batch_plan plan) {
  if (!plan) return SPPC_OK;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  if (plan->items) cudaFree(plan->items);
  if (plan->prefix) cudaFree(plan->prefix);
  if (plan->queue) cudaFree(plan->queue);
  delete plan;
  return SPPC_OK;
}

extern "C" sppc_status sppc_spmm_batch_plan(sppc_handle* handles, int32_t count, const double* const* X,
                                            double* const* Y, int32_t ncols, sppc_batch_plan* out) {
  using namespace sppc;
  if (!out || !handles || !X || !Y || count < 1 || count > 1024 || ncols < 1 || ncols > 8)
    return handle_fail(nullptr, SPPC_ERR_ARG, "sppc_spmm_batch_plan: bad arguments (1 <= count <= 1024, ncols <= 8)");
  *out = nullptr;
  const int kp = (ncols + 1) / 2 * 2;
  std::vector<BatchItem> items(count);
  std::vector<int64_t> prefix(count + 1, 0);
  std::vector<int64_t> rows(count);
  std::vector<float2*> t1(count), t2(count);
  for (int32_t i = 0; i < count; ++i) {
    if (!handles[i] || !X[i] || !Y[i]) return handle_fail(nullptr, SPPC_ERR_ARG, "sppc_spmm_batch_plan: NULL entry");
    int64_t n = 0;
    const SellDev* A = handle_matrix(handles[i], &n);
    if (A->nchunks != 1)
      return handle_fail(nullptr, SPPC_ERR_ARG, "sppc_spmm_batch_plan: matrices must use an untiled layout");
    if (A->f64)
      return handle_fail(nullptr, SPPC_ERR_ARG, "sppc_spmm_batch_plan: handles must use the double-float format");
    handle_scratch(handles[i], &t1[i], &t2[i]);
    items[i].A = *A;
    items[i].A.chunk_slice = nullptr;
    items[i].X = t1[i];
    items[i].Y = t2[i];
    rows[i] = n;
    prefix[i + 1] = prefix[i] + A->nslices;
  }
  sppc_batch_plan p = new sppc_batch_plan_s;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaMalloc(&p->items, sizeof(BatchItem) * count);
  if (e == cudaSuccess) e = cudaMalloc(&p->prefix, sizeof(int64_t) * (count + 1));
  if (e == cudaSuccess) e = cudaMalloc(&p->queue, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemcpy(p->items, items.data(), sizeof(BatchItem) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->prefix, prefix.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t ce = cudaSuccess;
    for (int32_t i = 0; i < count && ce == cudaSuccess; ++i) ce = f64_to_df(X[i], ncols, ncols, t1[i], kp, 0, rows[i], false, cs);
    if (ce == cudaSuccess) ce = spmm_batch(p->items, count, p->prefix, prefix[count], kp, p->queue, cs);
    for (int32_t i = 0; i < count && ce == cudaSuccess; ++i) ce = df_to_f64(t2[i], kp, Y[i], ncols, ncols, 0, rows[i], false, cs);
    e = cudaStreamEndCapture(cs, &p->graph);
    if (e == cudaSuccess) e = ce;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
  if (cs) cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    sppc_spmm_batch_destroy(p);
    return handle_fail(nullptr, SPPC_ERR_CUDA, cudaGetErrorString(e));
  }
  *out = p;
  return SPPC_OK;
}

extern "C" sppc_status sppc_spmm_batch_run(sppc_batch_plan plan, void* stream) {
  if (!plan || !plan->exec) return sppc::handle_fail(nullptr, SPPC_ERR_ARG, "sppc_spmm_batch_run: no plan");
  const cudaError_t e = cudaGraphLaunch(plan->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return sppc::handle_fail(nullptr, SPPC_ERR_CUDA, cudaGetErrorString(e));
  return SPPC_OK;
}
