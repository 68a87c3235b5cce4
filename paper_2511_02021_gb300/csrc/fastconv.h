// FP32 <-> FP64 conversions on the integer pipe.
//
// On this GPU a conversion between binary32 and binary64 issues on the FP64 pipe,
// which sustains 2 operations per SM per cycle against 64 for integer operations;
// in the mixed-precision column the conversions cost as much as the FP64 arithmetic
// they feed (measured: the lean column at R2B6/90 takes 12.2 ms per step with these
// helpers, 18.6 ms with the hardware conversions). These helpers build the result from
// the IEEE-754 encodings with integer operations (exponent re-bias, round to nearest
// even) instead, in as few instructions as the encodings allow.
// Ranges: the values of the dycore are finite and far from the binary32 limits;
// binary32 subnormals map to a signed zero, binary64 values below the binary32
// normal range to a signed zero, above it to infinity, NaN to infinity.
// icon_selftest() checks both against the hardware conversions.
#pragma once
#include <cuda_runtime.h>

namespace icon {

// exact: the exponent re-biased by one add on the magnitude shifted into place; infinities and
// NaNs re-biased twice (to 0x7ff), binary32 zeros and subnormals to a signed zero
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned a = u & 0x7fffffffu;
  unsigned h = (a >> 3) + 0x38000000u;                          // (1023 - 127) << 20
  if (a >= 0x7f800000u) h += 0x38000000u;
  const bool z = a < 0x00800000u;
  const unsigned hi = (u & 0x80000000u) | (z ? 0u : h);
  const unsigned lo = z ? 0u : (u << 29);
  return __hiloint2double((int)hi, (int)lo);
}

// round to nearest even: the top 9 exponent bits and 23 fraction bits shifted together out of
// the two words; in the binary32 normal range adding 2^30 turns the low 9 bits of the
// binary64 exponent into the binary32 exponent (e - 896 = e + 128 modulo 512) with a clear
// sign bit; the 29 dropped bits round up when above half, or at half with an odd result (a
// carry runs into the exponent, and out of the largest finite value exactly to infinity)
__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned hi = (unsigned)__double2hiint(d);
  const unsigned lo = (unsigned)__double2loint(d);
  const unsigned t = __funnelshift_l(lo, hi, 3) + 0x40000000u;
  const unsigned bits = t + (((lo & 0x1fffffffu) + 0x0fffffffu + (t & 1u)) >> 29);
  const unsigned ex = hi & 0x7ff00000u;
  const bool in_range = ex - 0x38100000u < 0x0fe00000u;         // binary64 exponent 897..1150
  const unsigned out = ex >= 0x47f00000u ? 0x7f800000u : 0u;    // overflow, infinities, NaNs; underflow
  return __uint_as_float((hi & 0x80000000u) | (in_range ? bits : out));
}

}  // namespace icon
