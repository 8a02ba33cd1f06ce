// Double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of two
// fp32 numbers with |lo| <= ulp(hi)/2, carrying ~48 significant bits.  All
// operations are built from the error-free transformations TwoSum (Knuth),
// Fast2Sum (Dekker, |a| >= |b|) and TwoProd via a fused multiply-add; they use
// the explicit-rounding intrinsics so the compiler never contracts or
// reassociates them.  FP64 on this GPU runs at ~1/70 of the FP32 rate, so the
// library computes its FP64-quality results this way on the FP32 pipes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sppc {

__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}

__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float e = __fsub_rn(b, __fsub_rn(s, a));
  return make_float2(s, e);
}

// Split of an FP64 value into hi + lo (both round-to-nearest conversions).
__device__ __forceinline__ float2 df_from_double(double x) {
  const float h = __double2float_rn(x);
  const float l = __double2float_rn(x - (double)h);
  return make_float2(h, l);
}

__device__ __forceinline__ double df_to_double(float2 a) { return (double)a.x + (double)a.y; }

__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float2 s = two_sum(a.x, b.x);
  const float2 t = two_sum(a.y, b.y);
  s.y = __fadd_rn(s.y, t.x);
  s = fast_two_sum(s.x, s.y);
  s.y = __fadd_rn(s.y, t.y);
  return fast_two_sum(s.x, s.y);
}

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ float2 df_sub(float2 a, float2 b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return fast_two_sum(p, e);
}

// a / b: fp32 quotient, remainder a - q1*b in double-float, corrected quotient.
__device__ __forceinline__ float2 df_div(float2 a, float2 b) {
  const float q1 = __fdiv_rn(a.x, b.x);
  const float2 r = df_sub(a, df_mul(make_float2(q1, 0.f), b));
  const float q2 = __fdiv_rn(r.x, b.x);
  return fast_two_sum(q1, q2);
}

// Accumulator (sh, sl): sh is the plain fp32 running sum, sl collects every
// rounding error exactly produced (TwoSum) plus the low-order product terms.
// sl is left unnormalised between calls; acc_norm() folds it back.
__device__ __forceinline__ void acc_mac(float& sh, float& sl, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float s = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}

// (sh, sl) += a (a df value)
__device__ __forceinline__ void acc_add(float& sh, float& sl, float2 a) {
  const float s = __fadd_rn(sh, a.x);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(a.x, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, a.y));
}

// Double-float multiply-add of one value v into two columns at once with packed
// f32x2 arithmetic: the same operations, in the same order and rounding, as two
// acc_mac calls (b - a is formed as fma(a, -1, b), rounded once like a
// subtraction), so the sums are bit-identical, in half the instructions.
__device__ __forceinline__ void acc_mac2(float2& sh, float2& sl, float2 v, float2 xc, float2 xd) {
  const float2 vh = make_float2(v.x, v.x), vl = make_float2(v.y, v.y);
  const float2 xh = make_float2(xc.x, xd.x), xl = make_float2(xc.y, xd.y);
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 p = __fmul2_rn(vh, xh);
  float2 e = __ffma2_rn(vh, xh, __fmul2_rn(p, m1));
  e = __ffma2_rn(vh, xl, e);
  e = __ffma2_rn(vl, xh, e);
  const float2 sn = __fadd2_rn(sh, p);
  const float2 bb = __ffma2_rn(sh, m1, sn);                        // sn - sh
  const float2 d1 = __ffma2_rn(__ffma2_rn(bb, m1, sn), m1, sh);    // sh - (sn - bb)
  const float2 d2 = __ffma2_rn(bb, m1, p);                         // p - bb
  sh = sn;
  sl = __fadd2_rn(sl, __fadd2_rn(__fadd2_rn(d1, d2), e));
}

__device__ __forceinline__ void acc_norm(float& sh, float& sl) {
  const float2 t = fast_two_sum(sh, sl);
  sh = t.x;
  sl = t.y;
}

__device__ __forceinline__ float2 acc_get(float sh, float sl) {
  const float2 t = two_sum(sh, sl);
  return t;
}

__device__ __forceinline__ float2 shfl_xor_df(float2 v, int m) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

__device__ __forceinline__ float2 warp_sum_df(float2 v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v = df_add(v, shfl_xor_df(v, m));
  return v;
}

}  // namespace sppc
