// Per-slice row sums of the SELL-16 SpMM, shared by the SpMM kernel and the
// persistent MINRES kernel.
#pragma once
#include "sppc_internal.h"
#include "val.cuh"

namespace sppc {

// L2 policy: keep lines (X rows are re-read by many matrix rows).
__device__ __forceinline__ uint64_t policy_keep() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// One lane's half of an X row: CPL double-float values starting at element
// `off` of row cidx.  A kp = 8 half row is one 256-bit load, so the two lanes of
// a row touch one 64-byte segment with a single L1 wavefront.  The rows are
// random and rarely reused inside an SM, so they bypass L1 allocation (letting
// them allocate cost 20-40% of the SpMM time on c2).
template <int KP>
__device__ __forceinline__ void gather_half(const float2* __restrict__ X, int cidx, int off, float2 (&x)[KP / 2],
                                            uint64_t pol) {
  const float2* p = X + static_cast<int64_t>(cidx) * KP + off;
  if constexpr (KP == 8) {
    float4 a, b;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p), "l"(pol));
    x[0] = make_float2(a.x, a.y);
    x[1] = make_float2(a.z, a.w);
    x[2] = make_float2(b.x, b.y);
    x[3] = make_float2(b.z, b.w);
  } else if constexpr (KP == 4) {
    float4 a;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w)
                 : "l"(p), "l"(pol));
    x[0] = make_float2(a.x, a.y);
    x[1] = make_float2(a.z, a.w);
  } else {
#pragma unroll
    for (int j = 0; j < KP / 2; ++j)
      asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;"
                   : "=f"(x[j].x), "=f"(x[j].y)
                   : "l"(p + j), "l"(pol));
  }
}

// Streamed matrix entries (read once): no L1 allocation.
__device__ __forceinline__ int ld_stream(const int32_t* p) {
  int v;
  asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float2 ld_stream(const float2* p) {
  float2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.f32 {%0,%1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
  return v;
}

// Row sums of slice s: lane pair (2*r, 2*r+1) owns row r of the slice, lane h
// of the pair accumulates columns [h*kp/2, (h+1)*kp/2) and returns them in out.
// Software pipeline of depth 2 per lane: the X half rows of entries t+1 and t+2
// are in flight while entry t is accumulated; the loop is unrolled by three so
// the three buffers rotate without register copies.  Entries are accumulated in
// order (double-float: renormalised after every 16th, whatever the unrolling);
// column pairs use the packed form (mac2), an odd last column the scalar one.
template <int KP, bool F64>
__device__ __forceinline__ void slice_rowsum(const SellDev& A, int64_t s, int rl, int off,
                                             const float2* __restrict__ X, uint64_t pol, float2 (&out)[KP / 2]) {
  using V = Ar<F64>;
  constexpr int CPL = KP / 2;
  constexpr int NP = CPL / 2;  // column pairs
  constexpr int H = kSliceH;
  const int64_t end = A.slice_ptr[s + 1];
  int64_t e = A.slice_ptr[s] + rl;
  typename V::Acc2 pa[NP > 0 ? NP : 1];
#pragma unroll
  for (int c = 0; c < NP; ++c) V::zero(pa[c]);
  typename V::Acc oa;  // odd last column
  V::zero(oa);
  float2 x0[CPL], x1[CPL], x2[CPL];
  float2 v0 = make_float2(0.f, 0.f), v1 = v0, v2 = v0;
  auto fetch = [&](int64_t ee, float2 (&x)[CPL], float2& v) {
    if (ee < end) {
      const int c = ld_stream(A.col + ee);
      v = ld_stream(A.val + ee);
      gather_half<KP>(X, c, off, x, pol);
    }
  };
  int cnt = 0;
  auto mac = [&](const float2 (&x)[CPL], float2 v) {
#pragma unroll
    for (int c = 0; c < NP; ++c) V::mac2(pa[c], v, x[2 * c], x[2 * c + 1]);
    if constexpr (CPL % 2 == 1) V::mac(oa, v, x[CPL - 1]);
    if (!F64 && ((++cnt) & 15) == 0) {
#pragma unroll
      for (int c = 0; c < NP; ++c) V::norm(pa[c]);
      if constexpr (CPL % 2 == 1) V::norm(oa);
    }
  };
  fetch(e, x0, v0);
  fetch(e + H, x1, v1);
  for (; e < end; e += 3 * H) {
    fetch(e + 2 * H, x2, v2);
    mac(x0, v0);
    if (e + H >= end) break;
    fetch(e + 3 * H, x0, v0);
    mac(x1, v1);
    if (e + 2 * H >= end) break;
    fetch(e + 4 * H, x1, v1);
    mac(x2, v2);
  }
#pragma unroll
  for (int c = 0; c < NP; ++c) {
    out[2 * c] = V::get0(pa[c]);
    out[2 * c + 1] = V::get1(pa[c]);
  }
  if constexpr (CPL % 2 == 1) out[CPL - 1] = V::get(oa);
}

}  // namespace sppc
