// FP32 <-> FP64 conversions on the integer pipe.
//
// On this GPU a conversion between binary32 and binary64 issues on the FP64 pipe,
// which sustains 2 operations per SM per cycle against 64 for integer operations;
// in the mixed-precision column the conversions cost as much as the FP64 arithmetic
// they feed. These helpers build the result from the IEEE-754 encodings with integer
// operations (field extraction, exponent re-bias, round to nearest even) instead.
// Ranges: the values of the dycore are finite and far from the binary32 limits;
// binary32 subnormals map to a signed zero, binary64 values below the binary32
// normal range to a signed zero, above it to infinity, NaN to infinity.
// icon_selftest() checks both against the hardware conversions.
#pragma once
#include <cuda_runtime.h>

namespace icon {

__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned m = u & 0x7fffffu;
  const unsigned e64 = (e == 0xffu) ? 0x7ffu : e + 896u;       // 1023 - 127
  const unsigned hi = (e == 0u) ? sign : (sign | (e64 << 20) | (m >> 3));
  const unsigned lo = (e == 0u) ? 0u : (m << 29);
  return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned hi = (unsigned)__double2hiint(d);
  const unsigned lo = (unsigned)__double2loint(d);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;              // binary32 biased exponent
  unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);            // top 23 of the 52 fraction bits
  const unsigned rest = lo & 0x1fffffffu;                      // the 29 dropped bits
  m += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  unsigned bits = ((unsigned)e << 23) + m;                     // a carry out of m bumps the exponent
  bits = (e <= 0) ? 0u : bits;
  bits = (e >= 255 || bits >= 0x7f800000u) ? 0x7f800000u : bits;
  return __uint_as_float(sign | bits);
}

}  // namespace icon
