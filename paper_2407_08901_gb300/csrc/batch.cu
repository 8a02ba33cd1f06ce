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
