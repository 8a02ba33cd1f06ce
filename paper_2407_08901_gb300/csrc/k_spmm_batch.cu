// Batched SpMM: Y_m = H_m X_m for many independent matrices (the batched
// workload: dozens of Hamiltonians of uneven sizes) in one persistent launch.
// The slices of all matrices form one global index space (prefix sums of the
// matrices' slice counts); warps take runs of slices from a device work queue
// (one atomic counter) until it is empty, so large and small matrices share the
// GPU without a launch per matrix or a tail per matrix.  Each slice is the same
// row sum as the single-matrix kernel (slice_rowsum), so the results are
// bit-identical to per-matrix products.  Untiled layouts only (one column tile:
// matrices of up to 1,310,720 columns).
#include "spmm_core.cuh"

namespace sppc {

namespace {

constexpr int kBatchGrab = 4;       // slices per work-queue grab (per warp)
constexpr int kMaxBatch = 1024;     // matrices per launch (prefix staged in shared memory)

template <int KP>
__global__ void __launch_bounds__(128, 7) k_spmm_batch(const BatchItem* __restrict__ items, int nitems,
                                                       const int64_t* __restrict__ prefix, int64_t total,
                                                       unsigned long long* __restrict__ queue) {
  constexpr int CPL = KP / 2;
  __shared__ int64_t sp[kMaxBatch + 1];
  for (int t = threadIdx.x; t <= nitems; t += blockDim.x) sp[t] = prefix[t];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int rl = lane >> 1;
  const int off = (lane & 1) * CPL;
  const uint64_t pol = policy_keep();
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(queue, static_cast<unsigned long long>(kBatchGrab));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= static_cast<unsigned long long>(total)) break;
    const int64_t g1 = min(static_cast<int64_t>(base) + kBatchGrab, total);
    for (int64_t g = static_cast<int64_t>(base); g < g1; ++g) {
      // matrix of global slice g: the last m with sp[m] <= g (binary search)
      int lo = 0, hi = nitems - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sp[mid] <= g) lo = mid;
        else hi = mid - 1;
      }
      const BatchItem& it = items[lo];
      const int64_t s = g - sp[lo];
      const int row = it.A.slice_rows[s * kSliceH + rl];
      float2 sum[CPL];
      slice_rowsum<KP, false>(it.A, s, rl, off, it.X, pol, sum);
      if (row < 0) continue;
      const int64_t b = static_cast<int64_t>(row) * KP + off;
#pragma unroll
      for (int c = 0; c < CPL; ++c) it.Y[b + c] = sum[c];
    }
  }
}

}  // namespace

cudaError_t spmm_batch(const BatchItem* items, int nitems, const int64_t* prefix, int64_t total, int kp,
                       unsigned long long* queue, cudaStream_t s) {
  if (nitems < 1 || nitems > kMaxBatch) return cudaErrorInvalidValue;
  if (total <= 0) return cudaSuccess;
  const void* fn = nullptr;
  switch (kp) {
    case 2: fn = reinterpret_cast<const void*>(k_spmm_batch<2>); break;
    case 4: fn = reinterpret_cast<const void*>(k_spmm_batch<4>); break;
    case 6: fn = reinterpret_cast<const void*>(k_spmm_batch<6>); break;
    case 8: fn = reinterpret_cast<const void*>(k_spmm_batch<8>); break;
    default: return cudaErrorInvalidValue;
  }
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, 128, 0);
  int64_t grid = static_cast<int64_t>(sms) * (per < 1 ? 1 : per);
  const int64_t need = (total + 4 * kBatchGrab - 1) / (4 * kBatchGrab);  // 4 warps per CTA
  if (grid > need) grid = need;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const unsigned g = static_cast<unsigned>(grid);
  switch (kp) {
    case 2: k_spmm_batch<2><<<g, 128, 0, s>>>(items, nitems, prefix, total, queue); break;
    case 4: k_spmm_batch<4><<<g, 128, 0, s>>>(items, nitems, prefix, total, queue); break;
    case 6: k_spmm_batch<6><<<g, 128, 0, s>>>(items, nitems, prefix, total, queue); break;
    default: k_spmm_batch<8><<<g, 128, 0, s>>>(items, nitems, prefix, total, queue); break;
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace sppc
