// fastmath.cuh -- low-latency FP64 reciprocal and reciprocal square root.
//
// On this GPU every dependent FP64 operation costs ~64 cycles -- additions,
// multiplications and fused multiply-adds, but also FP64<->FP32 conversions
// and FP64 comparisons -- and FP64 division or square root ~640 cycles,
// while FP32 and integer operations cost a few cycles.  The serial scalar
// work of the QR iteration (reflector generation, 2x2 rotations, swap
// factors) is a chain of such operations, so it uses:
//   - seeds from the FP32 approximate reciprocal / reciprocal square root,
//     with the FP32 operand and the FP64 seed assembled from the bit fields
//     by integer operations (no conversion instruction on the chain);
//   - one third-order Newton-Raphson step (the standard method, e.g.
//     Muller et al., "Handbook of Floating-Point Arithmetic", Sec. 5.3):
//       reciprocal:       e = 1 - a y,    y <- y + y (e + e^2)
//       rec. sqrt:        e = 1 - a y^2,  y <- y + y e (1/2 + 3e/8)
//     From the ~22-bit seed one step leaves a truncation error of order
//     2^-64, so results are within ~1 ulp of the correctly rounded FP64 value
//     (tested against CUDA's division and square root);
//   - integer tests of magnitudes and exponent ranges instead of FP64
//     comparisons.
// The seed is taken on the operand scaled by a power of two into [1, 4), so
// any normal operand with |exponent| <= 1000 works; other operands use IEEE
// division / sqrt.
#pragma once

#include <cuda_runtime.h>

// 2^k * x for an exponent adjustment that keeps x normal (bit manipulation).
__device__ __forceinline__ double fm_scale_pow2(double x, int k) {
  return __hiloint2double(__double2hiint(x) + (k << 20), __double2loint(x));
}

__device__ __forceinline__ int fm_exponent(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) - 1023; }

__device__ __forceinline__ float fm_rcp_approx_f32(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float fm_rsqrt_approx_f32(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// FP32 number 2^odd * (1.m) from the leading 23 mantissa bits of the double
// whose words are (hi, lo) (truncated; odd is 0 or 1).
__device__ __forceinline__ float fm_mantissa_f32(int hi, int lo, int odd) {
  unsigned fb = ((unsigned)(127 + odd) << 23) | (((unsigned)hi & 0xfffffu) << 3) | ((unsigned)lo >> 29);
  return __uint_as_float(fb);
}

// The double 2^s * f for a positive normal float f (exact, bit fields only).
__device__ __forceinline__ double fm_f32_to_f64_scaled(float f, int s) {
  unsigned fb = __float_as_uint(f);
  int fe = (int)((fb >> 23) & 0xffu) - 127;
  return __hiloint2double(((fe + s + 1023) << 20) | (int)((fb & 0x7fffffu) >> 3), (int)(fb << 29));
}

// 1/a for finite nonzero a.
__device__ __forceinline__ double fast_rcp(double a) {
  const int hi = __double2hiint(a);
  const int e = ((hi >> 20) & 0x7ff) - 1023;
  if (e < -1000 || e > 1000) return 1.0 / a;
  const float sf = fm_rcp_approx_f32(fm_mantissa_f32(hi, __double2loint(a), 0));   // 1 / (1.m)
  double y = fm_f32_to_f64_scaled(sf, -e);
  y = copysign(y, a);
  const double r = fma(-a, y, 1.0);
  const double p = fma(r, r, r);
  return fma(y, p, y);
}

// 1/sqrt(a) for finite a > 0.
__device__ __forceinline__ double fast_rsqrt(double a) {
  const int hi = __double2hiint(a);
  const int e = ((hi >> 20) & 0x7ff) - 1023;
  if (e < -1000 || e > 1000) return 1.0 / sqrt(a);
  const int k = e >> 1;                                                     // floor(e / 2)
  const float sf = fm_rsqrt_approx_f32(fm_mantissa_f32(hi, __double2loint(a), e & 1));  // (a 2^-2k)^-1/2
  const double y = fm_f32_to_f64_scaled(sf, -k);
  const double r = fma(-a * y, y, 1.0);
  const double ye = y * r;
  const double p = fma(0.375, r, 0.5);
  return fma(ye, p, y);
}

// |x| as an integer key: comparing keys of two doubles compares magnitudes
// (IEEE ordering of non-negative values) without an FP64 compare.
__device__ __forceinline__ long long fm_abs_key(double x) {
  return __double_as_longlong(x) & 0x7fffffffffffffffLL;
}

// |x| is zero or 2^-480 < |x| < 2^480 (up to the mantissa): the binary
// exponent e of x satisfies -480 < e < 480.  Integer operations only.
__device__ __forceinline__ bool fm_safe_exp(double x) {
  const unsigned hi = (unsigned)__double2hiint(x) & 0x7fffffffu;
  const unsigned be = hi >> 20;                        // biased exponent
  return ((hi | (unsigned)__double2loint(x)) == 0u) || (be - 544u <= 958u);
}

// true when every |x_i| is zero or has a binary exponent in (-480, 480), so
// that sums of squares neither overflow nor lose the smallest terms to
// underflow.
__device__ __forceinline__ bool fm_safe_range3(double x0, double x1, double x2) {
  return fm_safe_exp(x0) && fm_safe_exp(x1) && fm_safe_exp(x2);
}
