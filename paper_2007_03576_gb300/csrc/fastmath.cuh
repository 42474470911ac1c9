// fastmath.cuh -- low-latency FP64 reciprocal and reciprocal square root.
//
// On this GPU a dependent FP64 operation costs ~64 cycles and FP64 division
// or square root ~640 cycles, while FP32 and FP64<->FP32 conversions cost
// ~5 cycles.  The serial scalar work of the QR iteration (reflector
// generation, 2x2 rotations, swap factors) therefore uses Newton-Raphson
// iterations seeded from an FP32 approximation (the standard method, e.g.
// Muller et al., "Handbook of Floating-Point Arithmetic", Sec. 5.3):
//   reciprocal:      y <- y + y (1 - a y)          (quadratic convergence)
//   rec. sqrt:       y <- y + (y / 2) (1 - a y^2)
// Two steps from the ~23-bit FP32 seed give > 80 bits before the final
// rounding, so results are within ~1-2 ulp of the correctly rounded FP64
// value (tested against CUDA's division and square root).  The seed is taken
// on the operand scaled by a power of two into [1, 4), so any normal operand
// with |exponent| <= 1000 works; other operands use IEEE division / sqrt.
#pragma once

#include <cuda_runtime.h>

// 2^k * x for an exponent adjustment that keeps x normal (bit manipulation).
__device__ __forceinline__ double fm_scale_pow2(double x, int k) {
  return __hiloint2double(__double2hiint(x) + (k << 20), __double2loint(x));
}

__device__ __forceinline__ int fm_exponent(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) - 1023; }

// 1/a for finite nonzero a.
__device__ __forceinline__ double fast_rcp(double a) {
  int e = fm_exponent(a);
  if (e < -1000 || e > 1000) return 1.0 / a;
  double as = fm_scale_pow2(a, -e);                 // |as| in [1, 2)
  float f = __frcp_rn((float)as);                   // FP32 seed
  double y = fm_scale_pow2((double)f, -e);
  double r = fma(-a, y, 1.0);
  y = fma(y, r, y);
  r = fma(-a, y, 1.0);
  return fma(y, r, y);
}

// 1/sqrt(a) for finite a > 0.
__device__ __forceinline__ double fast_rsqrt(double a) {
  int e = fm_exponent(a);
  if (e < -1000 || e > 1000) return 1.0 / sqrt(a);
  int k = e >> 1;                                   // floor(e / 2)
  double as = fm_scale_pow2(a, -2 * k);             // as in [1, 4)
  float f = rsqrtf((float)as);                      // FP32 seed
  double y = fm_scale_pow2((double)f, -k);
  double h = 0.5 * y;
  double r = fma(-a * y, y, 1.0);
  y = fma(h, r, y);
  h = 0.5 * y;
  r = fma(-a * y, y, 1.0);
  return fma(h, r, y);
}

// |x| as an integer key: comparing keys of two doubles compares magnitudes
// (IEEE ordering of non-negative values) without an FP64 compare.
__device__ __forceinline__ long long fm_abs_key(double x) {
  return __double_as_longlong(x) & 0x7fffffffffffffffLL;
}

// true when every |x_i| lies in [2^-480, 2^480] or is zero, so that sums of
// squares neither overflow nor lose the smallest terms to underflow.
__device__ __forceinline__ bool fm_safe_range3(double x0, double x1, double x2) {
  int e0 = fm_exponent(x0), e1 = fm_exponent(x1), e2 = fm_exponent(x2);
  bool ok0 = (x0 == 0.0) || (e0 > -480 && e0 < 480);
  bool ok1 = (x1 == 0.0) || (e1 > -480 && e1 < 480);
  bool ok2 = (x2 == 0.0) || (e2 > -480 && e2 < 480);
  return ok0 && ok1 && ok2;
}
