// The two formats of the library's 8-byte value slots.
//
// Every vector, matrix value and coefficient on the device sits in an 8-byte
// slot typed float2.  A slot holds either a double-float pair hi + lo (about
// 48 significant bits, computed on the FP32 pipes; the default path) or the
// bits of one IEEE double (the native FP64 path, opts.precision = -1, computed
// with DFMA).  Kernels take the format as a template parameter and do their
// arithmetic through Ar<F64>: Ar<false> forwards to the error-free double-float
// operations of df.cuh, in the order the double-float kernels have always used;
// Ar<true> decodes the slot, uses correctly rounded FP64 operations (fused
// multiply-add for the accumulations) and encodes the result.  Both give a
// deterministic, fixed summation order.
#pragma once
#include "df.cuh"

namespace sppc {

// slot <-> double (bit reinterpretation: x carries the low word, y the high word)
__device__ __forceinline__ double slot_d(float2 v) {
  return __hiloint2double(__float_as_int(v.y), __float_as_int(v.x));
}
__device__ __forceinline__ float2 d_slot(double x) {
  return make_float2(__int_as_float(__double2loint(x)), __int_as_float(__double2hiint(x)));
}

template <bool F64>
struct Ar;

template <>
struct Ar<false> {
  struct Acc {
    float h, l;
  };
  struct Acc2 {  // two columns, packed f32x2
    float2 h, l;
  };
  static __device__ __forceinline__ void zero(Acc& a) { a.h = a.l = 0.f; }
  static __device__ __forceinline__ void zero(Acc2& a) { a.h = a.l = make_float2(0.f, 0.f); }
  static __device__ __forceinline__ void set(Acc& a, float2 v) {
    a.h = v.x;
    a.l = v.y;
  }
  static __device__ __forceinline__ void mac(Acc& a, float2 x, float2 y) { acc_mac(a.h, a.l, x, y); }
  static __device__ __forceinline__ void mac2(Acc2& a, float2 v, float2 xc, float2 xd) {
    acc_mac2(a.h, a.l, v, xc, xd);
  }
  static __device__ __forceinline__ void acc(Acc& a, float2 x) { acc_add(a.h, a.l, x); }
  static __device__ __forceinline__ void norm(Acc& a) { acc_norm(a.h, a.l); }
  static __device__ __forceinline__ void norm(Acc2& a) {
    acc_norm(a.h.x, a.l.x);
    acc_norm(a.h.y, a.l.y);
  }
  static __device__ __forceinline__ float2 get(const Acc& a) { return acc_get(a.h, a.l); }
  static __device__ __forceinline__ float2 get0(const Acc2& a) { return acc_get(a.h.x, a.l.x); }
  static __device__ __forceinline__ float2 get1(const Acc2& a) { return acc_get(a.h.y, a.l.y); }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return df_add(a, b); }
  static __device__ __forceinline__ float2 sub(float2 a, float2 b) { return df_sub(a, b); }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return df_mul(a, b); }
  static __device__ __forceinline__ float2 div(float2 a, float2 b) { return df_div(a, b); }
  static __device__ __forceinline__ float2 neg(float2 a) { return df_neg(a); }
  static __device__ __forceinline__ double to_d(float2 a) { return df_to_double(a); }
  static __device__ __forceinline__ float2 from_d(double x) { return df_from_double(x); }
  static __device__ __forceinline__ float2 one() { return make_float2(1.f, 0.f); }
  // the leading word, for sign and zero tests
  static __device__ __forceinline__ double lead(float2 a) { return (double)a.x; }
  // a denominator of magnitude below clamp becomes +-clamp (decided on the leading word)
  static __device__ __forceinline__ float2 clamp_den(float2 den, float clamp) {
    if (fabsf(den.x) < clamp) den = make_float2(den.x < 0.f ? -clamp : clamp, 0.f);
    return den;
  }
};

template <>
struct Ar<true> {
  struct Acc {
    double s;
  };
  struct Acc2 {
    double a, b;
  };
  static __device__ __forceinline__ void zero(Acc& a) { a.s = 0.0; }
  static __device__ __forceinline__ void zero(Acc2& a) { a.a = a.b = 0.0; }
  static __device__ __forceinline__ void set(Acc& a, float2 v) { a.s = slot_d(v); }
  static __device__ __forceinline__ void mac(Acc& a, float2 x, float2 y) { a.s = __fma_rn(slot_d(x), slot_d(y), a.s); }
  static __device__ __forceinline__ void mac2(Acc2& a, float2 v, float2 xc, float2 xd) {
    const double vv = slot_d(v);
    a.a = __fma_rn(vv, slot_d(xc), a.a);
    a.b = __fma_rn(vv, slot_d(xd), a.b);
  }
  static __device__ __forceinline__ void acc(Acc& a, float2 x) { a.s = __dadd_rn(a.s, slot_d(x)); }
  static __device__ __forceinline__ void norm(Acc&) {}
  static __device__ __forceinline__ void norm(Acc2&) {}
  static __device__ __forceinline__ float2 get(const Acc& a) { return d_slot(a.s); }
  static __device__ __forceinline__ float2 get0(const Acc2& a) { return d_slot(a.a); }
  static __device__ __forceinline__ float2 get1(const Acc2& a) { return d_slot(a.b); }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return d_slot(__dadd_rn(slot_d(a), slot_d(b))); }
  static __device__ __forceinline__ float2 sub(float2 a, float2 b) { return d_slot(__dsub_rn(slot_d(a), slot_d(b))); }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return d_slot(__dmul_rn(slot_d(a), slot_d(b))); }
  static __device__ __forceinline__ float2 div(float2 a, float2 b) { return d_slot(__ddiv_rn(slot_d(a), slot_d(b))); }
  static __device__ __forceinline__ float2 neg(float2 a) { return d_slot(-slot_d(a)); }
  static __device__ __forceinline__ double to_d(float2 a) { return slot_d(a); }
  static __device__ __forceinline__ float2 from_d(double x) { return d_slot(x); }
  static __device__ __forceinline__ float2 one() { return d_slot(1.0); }
  static __device__ __forceinline__ double lead(float2 a) { return slot_d(a); }
  static __device__ __forceinline__ float2 clamp_den(float2 den, float clamp) {
    double d = slot_d(den);
    if (fabs(d) < (double)clamp) d = d < 0.0 ? -(double)clamp : (double)clamp;
    return d_slot(d);
  }
};

// FP32 arithmetic on double-float slots: reads the leading word (the value
// rounded to FP32), writes (value, 0), a valid double-float slot.  Used by the
// FP32 small-space MINRES whose result iterative refinement corrects in
// double-float (or FP64).
struct ArF32 {
  struct Acc {
    float s;
  };
  static __device__ __forceinline__ void zero(Acc& a) { a.s = 0.f; }
  static __device__ __forceinline__ void set(Acc& a, float2 v) { a.s = v.x; }
  static __device__ __forceinline__ void mac(Acc& a, float2 x, float2 y) { a.s = __fmaf_rn(x.x, y.x, a.s); }
  static __device__ __forceinline__ void acc(Acc& a, float2 x) { a.s = __fadd_rn(a.s, x.x); }
  static __device__ __forceinline__ void norm(Acc&) {}
  static __device__ __forceinline__ float2 get(const Acc& a) { return make_float2(a.s, 0.f); }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return make_float2(__fadd_rn(a.x, b.x), 0.f); }
  static __device__ __forceinline__ float2 sub(float2 a, float2 b) { return make_float2(__fsub_rn(a.x, b.x), 0.f); }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return make_float2(__fmul_rn(a.x, b.x), 0.f); }
  static __device__ __forceinline__ float2 div(float2 a, float2 b) { return make_float2(__fdiv_rn(a.x, b.x), 0.f); }
  static __device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, 0.f); }
  static __device__ __forceinline__ double to_d(float2 a) { return (double)a.x; }
  static __device__ __forceinline__ float2 from_d(double x) { return make_float2(__double2float_rn(x), 0.f); }
  static __device__ __forceinline__ double lead(float2 a) { return (double)a.x; }
};

// Butterfly sum over the 32 lanes (fixed order).
template <bool F64>
__device__ __forceinline__ float2 warp_sum(float2 v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v = Ar<F64>::add(v, shfl_xor_df(v, m));
  return v;
}

// Value of a slot whose format is known only at run time (small driver kernels).
__device__ __forceinline__ double slot_get(float2 v, bool f64) { return f64 ? slot_d(v) : df_to_double(v); }
__device__ __forceinline__ float2 slot_put(double x, bool f64) { return f64 ? d_slot(x) : df_from_double(x); }

}  // namespace sppc
