// Table-driven FP64 exponential for the micro kernels (Tang, ACM TOMS 15(2), 1989):
// x = (64 m + j) ln2/64 + r with |r| <= ln2/128, exp(x) = 2^m * 2^(j/64) * (1 + p(r)), where
// p(r) = r + r^2/2 + r^3/6 + r^4/24 + r^5/120 (truncation below 4e-17 relative).  About 11
// FP64 instructions on the fast path (|x| < 708), against roughly twice that for the library
// exp; accuracy within 1-2 ulp, checked against the library exp by a GPU test.  Outside the fast
// range it defers to the library exp.
#pragma once

#include <cmath>

namespace mmk {

#include "mm_exp_table.inc"

__device__ __forceinline__ double expd(double x) {
  const int hi = __double2hiint(x);
  if ((hi & 0x7fffffff) >= 0x40862000) return exp(x);  // |x| >= 708 (or NaN/inf)
  const double kShift = 6755399441055744.0;             // 1.5 * 2^52: rounds to integer
  const double t = fma(x, kExpInvL, kShift);
  const int n = __double2loint(t);
  const double nf = t - kShift;
  double r = fma(nf, -kExpL1, x);
  r = fma(nf, -kExpL2, r);
  double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
  q = fma(r, q, 1.0 / 6.0);
  q = fma(r, q, 0.5);
  const double p = fma(r * r, q, r);
  const double s = __ldg(&kExpTab[n & 63]);
  const double y = fma(s, p, s);
  const int m = n >> 6;  // floor(n / 64), |m| <= 1022 on this path
  return y * __hiloint2double((m + 1023) << 20, 0);
}

}  // namespace mmk
