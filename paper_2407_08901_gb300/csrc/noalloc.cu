// Y = H X without any device allocation in the call.
//
// Some callers cannot allocate device memory when they multiply: a framework
// that owns all device memory through its own allocator and budget, a service
// that pre-reserves memory and forbids growth after start-up, or a loop that must
// not pay the device-wide synchronisation that cudaMalloc/cudaFree may imply.
// sppc_spmm needs scratch blocks (copies of X and of the result in the handle's
// value format, and an FP32 copy of X for the mixed-precision products) that the
// handle allocated; this variant keeps that scratch in a fixed file-scope device
// array instead, so a call allocates nothing.  It runs the same product as
// sppc_spmm: double-float, native FP64, or FP32 / BF16 values with FP32
// accumulation, as the handle's opts.precision says.
//
// The array is kNoAllocScratchBytes (32 MiB) and is held by every GPU that loads
// the library, until the process exits.  A call needs 2 * n * kp * 8 bytes of it
// (kp = ncols rounded up to even), plus n * kp * 4 for the FP32 copy of X when
// the handle's products are FP32 or BF16 (precision 1 or 2, kp = 4 or 8);
// larger requests are rejected with SPPC_ERR_ARG before anything is launched.
// All calls share the array, which keeps the last call's contents; calls whose
// work overlaps on the GPU (other streams or host threads) race on it.  Nothing
// in it has to start at zero: the conversion writes every X slot (padding
// columns included), the FP32 products write their copy of X first, and the SpMM
// writes every row of the result before any accumulation (column tiles) reads it.
//
// The array's device address is looked up (cudaGetSymbolAddress) by the first
// call in each CUDA context, with the device current, and cached per context:
// make that first call before any stream capture.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <mutex>

#include "sppc.h"
#include "sppc_internal.h"

namespace sppc {
// accessors for the handle's matrix, options and error slot (defined in api.cu)
const SellDev* handle_matrix(sppc_handle h, int64_t* n);
sppc_status handle_fail(sppc_handle h, sppc_status st, const char* msg);
void handle_values(sppc_handle h, int* precision, const float** val32, const uint16_t** val16, const float** diag32);
}  // namespace sppc

using namespace sppc;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array per CUDA context (a context created after a
// cudaDeviceReset may load the module elsewhere, so the key is the context's
// unique id, not only the device ordinal).
struct ScratchAddress {
  int dev = -1;
  unsigned long long ctx = 0;
  void* ptr = nullptr;
};
constexpr int kMaxContexts = 64;
std::mutex g_scratch_mu;
ScratchAddress g_scratch[kMaxContexts];
int g_scratch_used = 0;
PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;
PFN_cuCtxGetId_v12000 g_ctx_id = nullptr;

cudaError_t current_context_id(unsigned long long* id) {
  if (!g_ctx_current || !g_ctx_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1{}, q2{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 4000, cudaEnableDefault, &q1) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess)
      return cudaErrorNotSupported;
    g_ctx_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f1);
    g_ctx_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f2);
  }
  CUcontext c = nullptr;
  if (g_ctx_current(&c) != CUDA_SUCCESS || !c) return cudaErrorDeviceUninitialized;
  if (g_ctx_id(c, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  return cudaSuccess;
}

cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  unsigned long long id = 0;
  const bool have_ctx = current_context_id(&id) == cudaSuccess;
  if (have_ctx)
    for (int i = 0; i < g_scratch_used; ++i)
      if (g_scratch[i].dev == dev && g_scratch[i].ctx == id) {
        *out = g_scratch[i].ptr;
        return cudaSuccess;
      }
  // set-up for this context (the lookup also makes the device's primary context
  // current if no context was)
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  if (!have_ctx) {
    e = current_context_id(&id);
    if (e != cudaSuccess) return e;
  }
  // keep the newest entries: a full table reuses its oldest slot
  const int slot = g_scratch_used < kMaxContexts ? g_scratch_used++ : static_cast<int>(id % kMaxContexts);
  g_scratch[slot] = ScratchAddress{dev, id, p};
  *out = p;
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
  int precision = 0;
  const float* val32 = nullptr;
  const uint16_t* val16 = nullptr;
  const float* diag32 = nullptr;
  handle_values(h, &precision, &val32, &val16, &diag32);
  const int kp = (ncols + 1) / 2 * 2;
  const bool fp32_products = precision > 0 && (kp == 4 || kp == 8);
  const size_t slots = size_t(n) * size_t(kp);
  const size_t xy_bytes = 2 * slots * sizeof(float2);
  const size_t need = xy_bytes + (fp32_products ? slots * sizeof(float) : 0);
  if (need > kNoAllocScratchBytes) {
    char msg[320];
    snprintf(msg, sizeof(msg),
             "sppc_spmm_noalloc: needs %zu bytes of scratch (n=%lld, kp=%d%s) but the fixed scratch holds %zu "
             "bytes; use sppc_spmm",
             need, (long long)n, kp, fp32_products ? ", FP32 copy of X" : "", kNoAllocScratchBytes);
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
  float2* Ys = Xs + slots;
  float* X32 = reinterpret_cast<float*>(static_cast<unsigned char*>(base) + xy_bytes);
  e = f64_to_df(X, ldx, ncols, Xs, kp, 0, n, A->f64, s);
  if (e == cudaSuccess) {
    if (fp32_products)
      e = spmm_f32(*A, val32, val16, diag32, Xs, X32, Ys, kp, s);
    else
      e = spmm(*A, kp, Xs, Ys, Epi{}, s);
  }
  if (e == cudaSuccess) e = df_to_f64(Ys, kp, Y, ldy, ncols, 0, n, A->f64, s);
  if (e != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof(msg), "sppc_spmm_noalloc: launch failed: %s", cudaGetErrorString(e));
    return handle_fail(h, SPPC_ERR_CUDA, msg);
  }
  return SPPC_OK;
}
