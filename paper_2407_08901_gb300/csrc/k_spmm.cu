// SpMM Y = H X over the level-blocked SELL-32 layout, double-float arithmetic.
//
// The product with H is the dominant cost of SPPC: k SpMVs per order (paper
// Sec. 4.2-4.3), plus the products with the leading block H0_hat inside the
// small solves.  One warp owns a 32-row slice, one lane one row, so the row
// reduction needs no shuffles; the 32 lanes' t-th entries are contiguous, so
// column indices (4 B) and double-float values (8 B) stream in fully coalesced
// 128 B / 256 B transactions with an evict-first hint (they are read once).
// Each entry gathers one row of X (kp double-float values, 16-64 B, 16 B
// aligned) through the read-only path; slices follow the level order, so a
// wave of warps gathers from one window of levels of X, which stays in L2.
#include "df.cuh"
#include "sppc_internal.h"

namespace sppc {

namespace {

template <int KP>
__device__ __forceinline__ void gather_row(const float2* __restrict__ X, int cidx, float4 (&x)[KP / 2]) {
  const float4* xr = reinterpret_cast<const float4*>(X + static_cast<int64_t>(cidx) * KP);
#pragma unroll
  for (int q = 0; q < KP / 2; ++q) x[q] = __ldg(xr + q);
}

// Software pipeline per lane: the column index / value of entry t+2 and the X
// row of entry t+1 are in flight while entry t is multiplied and accumulated.
// All lanes of a slice run the same number of steps (the slice width).
template <int KP>
__global__ void __launch_bounds__(128) k_spmm_sell(SellDev A, const float2* __restrict__ X, float2* __restrict__ Y,
                                                   Epi epi) {
  static_assert(KP % 2 == 0 && KP <= 8, "kp must be 2, 4, 6 or 8");
  const int lane = threadIdx.x & 31;
  const int64_t gw = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t s = gw; s < A.nslices; s += nw) {
    const int64_t beg = A.slice_ptr[s];
    const int64_t end = A.slice_ptr[s + 1];
    const int row = A.slice_rows[s * 32 + lane];
    float ah[KP], al[KP];
#pragma unroll
    for (int c = 0; c < KP; ++c) ah[c] = al[c] = 0.f;
    int64_t e = beg + lane;
    float4 x0[KP / 2];
    float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
    int c1 = 0;
    if (e < end) {
      const int c0 = __ldcs(A.col + e);
      v0 = __ldcs(A.val + e);
      gather_row<KP>(X, c0, x0);
      if (e + 32 < end) {
        c1 = __ldcs(A.col + e + 32);
        v1 = __ldcs(A.val + e + 32);
      }
    }
    int cnt = 0;
    for (; e < end; e += 32) {
      float4 x1[KP / 2];
      const bool more1 = (e + 32 < end);
      if (more1) gather_row<KP>(X, c1, x1);
      int c2 = 0;
      float2 v2 = make_float2(0.f, 0.f);
      if (e + 64 < end) {
        c2 = __ldcs(A.col + e + 64);
        v2 = __ldcs(A.val + e + 64);
      }
#pragma unroll
      for (int q = 0; q < KP / 2; ++q) {
        acc_mac(ah[2 * q], al[2 * q], v0, make_float2(x0[q].x, x0[q].y));
        acc_mac(ah[2 * q + 1], al[2 * q + 1], v0, make_float2(x0[q].z, x0[q].w));
      }
      if (((++cnt) & 15) == 0) {
#pragma unroll
        for (int c = 0; c < KP; ++c) acc_norm(ah[c], al[c]);
      }
      if (more1) {
#pragma unroll
        for (int q = 0; q < KP / 2; ++q) x0[q] = x1[q];
      }
      v0 = v1;
      v1 = v2;
      c1 = c2;
    }
    if (row < 0) continue;
    const int64_t base = static_cast<int64_t>(row) * KP;
#pragma unroll
    for (int c = 0; c < KP; ++c) {
      float2 r = acc_get(ah[c], al[c]);
      if (epi.alpha) r = df_mul(epi.alpha[c], r);
      if (epi.beta) r = df_add(r, df_mul(epi.beta[c], X[base + c]));
      if (epi.gamma) r = df_add(r, df_mul(epi.gamma[c], epi.Z[base + c]));
      Y[base + c] = r;
    }
  }
}

int g_grid = 0;

}  // namespace

int spmm_default_grid() {
  if (g_grid == 0) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spmm_sell<8>, 128, 0);
    if (per_sm < 1) per_sm = 1;
    g_grid = sms * per_sm;
  }
  return g_grid;
}

cudaError_t spmm(const SellDev& A, int kp, const float2* X, float2* Y, const Epi& epi, cudaStream_t s) {
  if (A.nslices == 0) return cudaSuccess;
  const int64_t warps_needed = A.nslices;
  int64_t grid = (warps_needed + 3) / 4;
  const int64_t gmax = spmm_default_grid();
  if (grid > gmax) grid = gmax;
  switch (kp) {
    case 2: k_spmm_sell<2><<<(unsigned)grid, 128, 0, s>>>(A, X, Y, epi); break;
    case 4: k_spmm_sell<4><<<(unsigned)grid, 128, 0, s>>>(A, X, Y, epi); break;
    case 6: k_spmm_sell<6><<<(unsigned)grid, 128, 0, s>>>(A, X, Y, epi); break;
    case 8: k_spmm_sell<8><<<(unsigned)grid, 128, 0, s>>>(A, X, Y, epi); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace sppc
