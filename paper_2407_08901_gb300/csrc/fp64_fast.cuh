// Fast FP64 reciprocal and reciprocal square root for serial scalar chains.
#pragma once

namespace sppc {

// On this GPU an FP64 division costs about 430 cycles and a square root about
// 680, against 64 for a dependent FP64 multiply-add, so serial scalar chains
// (Householder reflectors, tridiagonal solves) take 1/x and 1/sqrt(x) from the
// hardware approximations (relative error below 2^-20) and one third-order
// correction: with e = 1 - x r, 1/x = r (1 + e + e^2 + ...); with e = 1 - x y^2,
// 1/sqrt(x) = y (1 + e/2 + 3e^2/8 + ...).  The truncated series leave a relative
// error below 2^-57, so the results are within a few ulps (not correctly
// rounded).  Values of extreme magnitude (exponent within 64 of either end of
// the range) take the IEEE operations.
__device__ __forceinline__ bool mid_range64(double x) {
  const int ex = (__double2hiint(x) >> 20) & 0x7FF;
  return ex > 64 && ex < 2046 - 64;
}
__device__ __forceinline__ double recip64(double x) {
  if (!mid_range64(x)) return 1.0 / x;
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  const double e = __fma_rn(-x, r, 1.0);
  return __fma_rn(r, __fma_rn(e, e, e), r);
}
__device__ __forceinline__ double rsqrt64(double x) {
  if (!mid_range64(x)) return 1.0 / sqrt(x);
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = __fma_rn(-__dmul_rn(x, y), y, 1.0);
  return __fma_rn(__dmul_rn(y, e), __fma_rn(e, 0.375, 0.5), y);
}
// sqrt(x) for x >= 0 (0 for x = 0) as x / sqrt(x)
__device__ __forceinline__ double sqrt64(double x) { return x > 0.0 ? x * rsqrt64(x) : 0.0; }

}  // namespace sppc
