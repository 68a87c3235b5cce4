// FP64 reciprocal by Newton-Raphson refinement of a binary32 seed.
//
// An IEEE FP64 division issues about eight FP64-pipe operations on this GPU, whose
// FP64 pipe retires one warp instruction per SM every 16 cycles; the column solves
// divide once or more per level. recip64 needs three FP64 FMAs:
//   seed   y0 = rcp.approx.ftz.f32 of x rounded to binary32 (relative error below
//          2^-22 including the rounding of x; the conversions run on the integer pipe),
//   e      = 1 - x y0                         (one FMA, nearly exact),
//   1/x    = y0 / (1 - e) = y0 (1 + e + e^2 + e^3 + ...), truncated after e^2:
//   y      = y0 + y0 (e + e^2)                (two FMAs).
// The truncation leaves a relative error of order e^3 < 2^-66, so the result is within
// one ulp of 1/x (third-order Newton-Raphson step; P. Markstein, "Computation of
// elementary functions on the IBM RISC System/6000 processor", IBM J. Res. Dev. 34(1),
// 1990). Domain: finite |x| in [2^-125, 2^125] (the dycore's divisors are densities,
// potential temperatures and pivots of a diagonally dominant matrix); outside it the
// binary32 seed is zero or infinite and the result is not finite, which the column
// kernels' finiteness checks report. icon_selftest() compares recip64 and x * recip64
// with the hardware division.
#pragma once
#include <cuda_runtime.h>

#include "fastconv.h"

namespace icon {

__device__ __forceinline__ double recip64(double x) {
  const float xs = f64_to_f32(x);
  float ys;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ys) : "f"(xs));
  const double y0 = f32_to_f64(ys);
  const double e = fma(-x, y0, 1.0);
  const double t = fma(e, e, e);
  return fma(y0, t, y0);
}

}  // namespace icon
