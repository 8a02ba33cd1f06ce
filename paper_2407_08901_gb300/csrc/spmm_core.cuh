// Per-slice row sums of the SELL-16 SpMM, shared by the SpMM kernel and the
// persistent MINRES kernel.
#pragma once
#include "df.cuh"
#include "sppc_internal.h"

namespace sppc {

// L2 policy: keep lines (X rows are re-read by many matrix rows).
__device__ __forceinline__ uint64_t policy_keep() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// One lane's half of an X row: CPL double-float values starting at element
// `off` of row cidx.  A kp = 8 half row is one 256-bit load, so the two lanes of
// a row touch one 64-byte segment with a single L1 wavefront.
template <int KP>
__device__ __forceinline__ void gather_half(const float2* __restrict__ X, int cidx, int off, float2 (&x)[KP / 2],
                                            uint64_t pol) {
  const float2* p = X + static_cast<int64_t>(cidx) * KP + off;
  if constexpr (KP == 8) {
    float4 a, b;
    asm volatile("ld.global.nc.L2::cache_hint.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p), "l"(pol));
    x[0] = make_float2(a.x, a.y);
    x[1] = make_float2(a.z, a.w);
    x[2] = make_float2(b.x, b.y);
    x[3] = make_float2(b.z, b.w);
  } else if constexpr (KP == 4) {
    float4 a;
    asm volatile("ld.global.nc.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w)
                 : "l"(p), "l"(pol));
    x[0] = make_float2(a.x, a.y);
    x[1] = make_float2(a.z, a.w);
  } else {
#pragma unroll
    for (int j = 0; j < KP / 2; ++j) x[j] = __ldg(p + j);
  }
}

// Row sums of slice s: lane pair (2*r, 2*r+1) owns row r of the slice, lane h
// of the pair accumulates columns [h*kp/2, (h+1)*kp/2) into (ah, al).  Software
// pipeline per lane: the column index / value of entry t+2 and the half row of
// X for entry t+1 are in flight while entry t is multiplied and accumulated.
// All lanes of a slice run the same number of steps (the slice width).
template <int KP>
__device__ __forceinline__ void slice_rowsum(const SellDev& A, int64_t s, int rl, int off,
                                             const float2* __restrict__ X, uint64_t pol, float (&ah)[KP / 2],
                                             float (&al)[KP / 2]) {
  constexpr int CPL = KP / 2;
  constexpr int H = kSliceH;
  const int64_t end = A.slice_ptr[s + 1];
  int64_t e = A.slice_ptr[s] + rl;
#pragma unroll
  for (int c = 0; c < CPL; ++c) ah[c] = al[c] = 0.f;
  float2 x0[CPL];
  float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
  int c1 = 0;
  if (e < end) {
    const int c0 = __ldcs(A.col + e);
    v0 = __ldcs(A.val + e);
    gather_half<KP>(X, c0, off, x0, pol);
    if (e + H < end) {
      c1 = __ldcs(A.col + e + H);
      v1 = __ldcs(A.val + e + H);
    }
  }
  int cnt = 0;
  for (; e < end; e += H) {
    float2 x1[CPL];
    const bool more1 = (e + H < end);
    if (more1) gather_half<KP>(X, c1, off, x1, pol);
    int c2 = 0;
    float2 v2 = make_float2(0.f, 0.f);
    if (e + 2 * H < end) {
      c2 = __ldcs(A.col + e + 2 * H);
      v2 = __ldcs(A.val + e + 2 * H);
    }
#pragma unroll
    for (int c = 0; c < CPL; ++c) acc_mac(ah[c], al[c], v0, x0[c]);
    if (((++cnt) & 15) == 0) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) acc_norm(ah[c], al[c]);
    }
    if (more1) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) x0[c] = x1[c];
    }
    v0 = v1;
    v1 = v2;
    c1 = c2;
  }
}

}  // namespace sppc
