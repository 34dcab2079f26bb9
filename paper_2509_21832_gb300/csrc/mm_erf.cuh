// FP64 error function for the KFVS half fluxes (Section 5.4): on |x| < 1.5, where the normal
// velocity is below about 1.5 sqrt(2 T) (the usual case), erf(x) = x P(x^2) with P the
// degree-14 polynomial of mm_erf_poly.inc (interpolant of erf(sqrt(s))/sqrt(s) at Chebyshev
// nodes of [0, 2.25], from the Maclaurin series; written by gen_erf_poly.py): 16 FP64
// instructions, within 2.6e-16 relative of erf (about 2.3 ulp at most; a GPU test bounds its
// distance from the library erf by 5 ulp).  Elsewhere, and for NaN, the library erf.
#pragma once

#include <cmath>

namespace mmk {

#include "mm_erf_poly.inc"

__device__ __forceinline__ double erfd(double x) {
  if (fabs(x) < 1.5) return x * erf_poly(x * x);
  return erf(x);
}

}  // namespace mmk
