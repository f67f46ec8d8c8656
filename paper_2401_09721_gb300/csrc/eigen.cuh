// Pieces of the eigen step of the noise estimate (Section 2.3) that the
// window-1 kernel and the wider-window kernels share: the Jacobi rotation of
// one pair, a float64 quotient without the library division, order keys of
// float64 values, and the threshold below which an eigenvalue is zero.
#pragma once

#include "fgbd_internal.cuh"

namespace fgbd {
namespace {

constexpr double kZeroEigRel = 1e-9;  // relative size below which an eigenvalue is zero

// The rotation of the pair p < q that zeroes a_pq, as the columns of J for p
// and for q: (c, -s) and (c, s).  cos 2phi = |a_qq - a_pp| / r with r =
// sqrt((a_qq - a_pp)^2 + 4 a_pq^2), c = sqrt((1 + cos 2phi) / 2), |s| =
// |a_pq| / (r c), and s takes the sign of (a_qq - a_pp) a_pq (the smaller of
// the two angles that zero a_pq).  A pair with |a_pq| <= thr is not rotated.
__device__ __forceinline__ void jacobi_rotation(float app, float aqq, float apq, float thr, float2& cp, float2& cq) {
  cp = cq = make_float2(1.f, 0.f);
  if (!(fabsf(apq) > thr)) return;
  const float tau = aqq - app;
  const float two_a = 2.f * apq;
  const float rr = rsqrtf(fmaf(tau, tau, two_a * two_a));
  const float h = fmaf(0.5f * fabsf(tau), rr, 0.5f);
  const float ic = rsqrtf(h);
  const float c = h * ic;
  float s = fabsf(apq) * rr * ic;
  if ((tau < 0.f) != (apq < 0.f)) s = -s;
  cp = make_float2(c, -s);
  cq = make_float2(c, s);
}

// a / b in float64 from a float32 reciprocal and Newton steps (fused
// multiply-adds only; the library division is much longer on this GPU).
// Within an ulp or two of the rounded quotient for b > 0.
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
