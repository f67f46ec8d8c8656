// Pieces of the eigen step of the noise estimate (Section 2.3) that the
// window-1 kernel and the wider-window kernels share: the Jacobi rotation of
// one pair, the eigenvectors of a 3x3 colour covariance (the warm start), a
// float64 quotient without the library division, order keys of float64
// values, and the threshold below which an eigenvalue is zero.
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

// Eigenvectors of the symmetric 3x3 matrix m (in place: its columns on
// return), by cyclic Jacobi in float32 (a few sweeps converge for 3x3).
__device__ __noinline__ void colour_basis(float (*m)[3]) {
  float a[3][3], v[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      a[i][j] = m[i][j];
      v[i][j] = i == j ? 1.f : 0.f;
    }
  const float scale = fabsf(a[0][0]) + fabsf(a[1][1]) + fabsf(a[2][2]);
  for (int sweep = 0; sweep < 8; ++sweep) {
    if (!(fabsf(a[0][1]) + fabsf(a[0][2]) + fabsf(a[1][2]) > 1e-7f * scale)) break;
    for (int pair = 0; pair < 3; ++pair) {
      const int p = pair == 2 ? 1 : 0, q = pair == 0 ? 1 : 2;
      float2 cp, cq;
      jacobi_rotation(a[p][p], a[q][q], a[p][q], 1e-7f * scale, cp, cq);
      const float c = cp.x, s = cq.y;  // column p = (c, -s) at rows (p, q), column q = (s, c)
      if (s == 0.f) continue;
      for (int k = 0; k < 3; ++k) {  // A J
        const float akp = a[k][p], akq = a[k][q];
        a[k][p] = c * akp - s * akq;
        a[k][q] = s * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) {  // J^T A
        const float apk = a[p][k], aqk = a[q][k];
        a[p][k] = c * apk - s * aqk;
        a[q][k] = s * apk + c * aqk;
      }
      for (int k = 0; k < 3; ++k) {  // V J
        const float vkp = v[k][p], vkq = v[k][q];
        v[k][p] = c * vkp - s * vkq;
        v[k][q] = s * vkp + c * vkq;
      }
    }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) m[i][j] = v[i][j];
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
