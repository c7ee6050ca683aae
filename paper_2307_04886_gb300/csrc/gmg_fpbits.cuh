// Floating-point conversions and tests done on the IEEE 754 bit patterns
// with integer operations.
//
// On GB300 the FP64 pipe of an SM sub-partition takes 64 cycles per warp
// instruction and a conversion between FP64 and FP32 about 96 (measured), so
// in the set-up and CG kernels, where every row converts a value, the
// conversions and FP64 comparisons, not the memory traffic, bound the time.
// The integer pipe does the same work in a few cycles.  Each helper gives the
// bits the IEEE 754 operation defines (round to nearest, ties to even, for
// the narrowing conversion); values outside the ranges handled on the bits
// (subnormal results, infinities, NaN) go to the hardware conversion, which
// is rare in this code and gives the same definition.
#pragma once

#include <cstdint>

namespace gmg {

// float(x), round to nearest even.  Handled on the bits when the result is a
// normal float (double exponent 897..1150, carry into the exponent included,
// so a value past the largest float rounds to infinity as it must).
__device__ __forceinline__ float f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned ex = (unsigned)(b >> 52) & 0x7FFu;
  if (ex - 897u > 253u) return (float)x;
  unsigned r = ((ex - 896u) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu);
  const unsigned rem = (unsigned)(b & 0x1FFFFFFFu);  // the 29 bits rounded away
  r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
  return __uint_as_float(r | ((unsigned)(b >> 32) & 0x80000000u));
}

// double(f), exact: normal floats and zeros on the bits.
__device__ __forceinline__ double f64_of(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFFu;
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  if ((u & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)s);
  if (e == 0u || e == 0xFFu) return (double)f;
  return __longlong_as_double(
      (long long)(s | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

__device__ __forceinline__ double to_f64(float f) { return f64_of(f); }
__device__ __forceinline__ double to_f64(double x) { return x; }

// x is neither infinite nor NaN.
__device__ __forceinline__ bool finite_bits(double x) {
  return ((unsigned long long)__double_as_longlong(x) >> 52 & 0x7FFu) != 0x7FFu;
}

// x > 0 and finite.
__device__ __forceinline__ bool positive_bits(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b < 0x7FF0000000000000LL;
}

// 1 / d within one unit in the last place: an FP32 seed r0 built from d's
// exponent and leading 23 mantissa bits and widened exactly (relative error
// e0 = 1 - d r0 of about 2^-22), then one cubic Newton-Raphson step
// r = r0 (1 + e0 + e0^2), whose truncation error is e0^3 (about 2^-66).
// |d| outside [2^-100, 2^101) uses the FP64 division.
__device__ __forceinline__ double recip_newton(double d) {
  const long long bits = __double_as_longlong(d);
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex < 1023 - 100 || ex > 1023 + 100) return 1.0 / d;
  const unsigned fb = ((unsigned)((unsigned long long)bits >> 32) & 0x80000000u) | ((unsigned)(ex - 1023 + 127) << 23) |
                      ((unsigned)(bits >> 29) & 0x7FFFFFu);
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(__uint_as_float(fb)));
  const double r0 = f64_of(rf);
  const double e0 = __fma_rn(-d, r0, 1.0);
  const double t = __fma_rn(e0, e0, e0);
  return __fma_rn(r0, t, r0);
}

}  // namespace gmg
