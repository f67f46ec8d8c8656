// Pieces of the eigen step of the noise estimate (Section 2.3) that the
// window-1 kernel and the wider-window kernels share: a float64 quotient
// without the library division, order keys of float64 values, and the
// threshold below which an eigenvalue is zero.
#pragma once

#include "fgbd_internal.cuh"

namespace fgbd {
namespace {

constexpr double kZeroEigRel = 1e-9;  // relative size below which an eigenvalue is zero

// a / b in float64 from a float32 reciprocal and Newton steps (fused
// multiply-adds only; the library division is much longer on this GPU).
// The method is Newton-Raphson for 1/b: r <- r + r (1 - b r) doubles the
// correct bits of a float32 seed (24 -> 48 -> ~53), then one residual
// correction of the quotient, q + r (a - b q).  Within an ulp or two of the
// rounded quotient for b > 0 in float32's normal range (tested against CUDA's
// division by fgbd_debug_div).
__device__ __forceinline__ double div_newton(double a, double b) {
  double r = double(__frcp_rn(float(b)));
  r = fma(r, fma(-b, r, 1.0), r);
  r = fma(r, fma(-b, r, 1.0), r);
  const double q = a * r;
  return fma(r, fma(-b, q, a), q);
}

// 64-bit integer whose signed order is the numeric order of the double x
__device__ __forceinline__ long long order_key(double x) {
  const long long b = __double_as_longlong(x);
  return b < 0 ? (b ^ 0x7fffffffffffffffLL) : b;
}

}  // namespace
}  // namespace fgbd
