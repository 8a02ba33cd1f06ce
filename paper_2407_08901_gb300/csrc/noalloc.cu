// Y = H X without any device allocation in the call.
//
// Some callers cannot allocate device memory when they multiply: a framework
// that owns all device memory through its own allocator and budget, a service
// that pre-reserves memory and forbids growth after start-up, or a loop that must
// not pay the device-wide synchronisation that cudaMalloc/cudaFree may imply.
// sppc_spmm needs two scratch blocks (double-float copies of X and of the result)
// that the handle allocated; this variant keeps that scratch in a fixed
// file-scope device array instead, so a call allocates nothing.
//
// The array is kNoAllocScratchBytes (32 MiB) and is held by every GPU that loads
// the library, until the process exits.  A call needs 2 * n * kp * 8 bytes of it
// (kp = ncols rounded up to even), i.e. n * kp <= 2,097,152; larger requests are
// rejected with SPPC_ERR_ARG before anything is launched.  All calls share the
// array, which keeps the last call's contents; calls whose work overlaps on the
// GPU (other streams or host threads) race on it.  Nothing in it has to start at
// zero: the conversion writes every X slot (padding columns included) and the
// SpMM writes every row of the result before any accumulation reads it.
#include <cstdio>
#include <mutex>

#include "sppc.h"
#include "sppc_internal.h"

namespace sppc {
// accessors for the handle's matrix and error slot (defined in api.cu)
const SellDev* handle_matrix(sppc_handle h, int64_t* n);
sppc_status handle_fail(sppc_handle h, sppc_status st, const char* msg);
}  // namespace sppc

using namespace sppc;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array, resolved once per device with that device current.
struct ScratchAddress {
  bool ready = false;
  void* ptr = nullptr;
};
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
ScratchAddress g_scratch[kMaxDevices];

cudaError_t scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch[dev].ready) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch[dev].ptr = p;
    g_scratch[dev].ready = true;
  }
  *out = g_scratch[dev].ptr;
  return cudaSuccess;
}

}  // namespace

extern "C" sppc_status sppc_spmm_noalloc(sppc_handle h, const double* X, int64_t ldx, double* Y, int64_t ldy,
                                         int32_t ncols, void* stream) {
  if (!h) return handle_fail(nullptr, SPPC_ERR_ARG, "sppc_spmm_noalloc: NULL handle");
  if (!X || !Y || ncols < 1 || ncols > 8 || ldx < ncols || ldy < ncols)
    return handle_fail(h, SPPC_ERR_ARG, "sppc_spmm_noalloc: bad arguments (ncols in [1,8], ld >= ncols)");
  int64_t n = 0;
  const SellDev* A = handle_matrix(h, &n);
  const int kp = (ncols + 1) / 2 * 2;
  const size_t need = size_t(2) * size_t(n) * size_t(kp) * sizeof(float2);
  if (need > kNoAllocScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof(msg),
             "sppc_spmm_noalloc: needs %zu bytes of scratch (2*n*kp*8 with n=%lld, kp=%d) but the fixed scratch "
             "holds %zu bytes (n*kp <= %zu); use sppc_spmm",
             need, (long long)n, kp, kNoAllocScratchBytes, kNoAllocScratchBytes / (2 * sizeof(float2)));
    return handle_fail(h, SPPC_ERR_ARG, msg);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  void* base = nullptr;
  if (e == cudaSuccess) e = scratch_address(dev, &base);
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof(msg), "sppc_spmm_noalloc: scratch address: %s", cudaGetErrorString(e));
    return handle_fail(h, SPPC_ERR_CUDA, msg);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float2* Xs = static_cast<float2*>(base);
  float2* Ys = Xs + n * kp;
  e = f64_to_df(X, ldx, ncols, Xs, kp, 0, n, s);
  if (e == cudaSuccess) e = spmm(*A, kp, Xs, Ys, Epi{}, s);
  if (e == cudaSuccess) e = df_to_f64(Ys, kp, Y, ldy, ncols, 0, n, s);
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof(msg), "sppc_spmm_noalloc: launch failed: %s", cudaGetErrorString(e));
    return handle_fail(h, SPPC_ERR_CUDA, msg);
  }
  return SPPC_OK;
}
