// Eigenvector estimates of the patch covariance for the noise estimate
// (Section 2.3), which needs the eigenvalues only.
//
// The eigenvalues themselves are the float64 Rayleigh quotients
// v^T Sigma v / v^T v of the vectors computed here (done by the caller): their
// error is second order in the vector error, so float32 vectors give
// eigenvalues far inside the noise estimate's tolerance.  The vectors come
// from the textbook route for a small dense symmetric matrix, in float32:
//   1. Householder reduction to tridiagonal form T = Q^T A Q (D - 2
//      reflections H_k = I - u_k u_k^T / h_k), the rows of A in registers:
//      for D <= 32 spread over the block's warps (lane j holds column j), so
//      the products of each step are warp reductions side by side; for
//      larger D in one warp;
//   2. the eigenvalues of T by Sturm-count multisection (every participating
//      thread counts at its own point, so each pass narrows every bracket at
//      once; no iteration depends on convergence);
//   3. one eigenvector of T per eigenvalue by two steps of inverse iteration
//      (an LDL^T solve of T - mu I), one thread each;
//   4. back to A's basis: v = H_0 H_1 ... H_{D-3} z.
// Within a cluster of eigenvalues closer than float32 resolution the vectors
// may mix, but each quotient then lies inside the cluster, so the eigenvalues
// stay within the cluster's width.  If a quotient is not finite the caller
// falls back to the multisection value, which is within float32 resolution.
#pragma once

#include "fgbd_internal.cuh"

namespace fgbd {
namespace {

// Shared-memory workspace of eig_vectors_f32<D, NT>.
template <int D, int NT>
struct TridiagSmem {
  static constexpr int kPer = NT / D;  // multisection points per eigenvalue and pass
  float U[D > 2 ? D - 2 : 1][D];       // reflection vectors u_k (rows)
  float h[D];                          // and their h_k = |u_k|^2 / 2 (0: no reflection)
  float d[D], e[D], e2[D];             // T: diagonal, off-diagonal e_i = T[i][i+1], e_i^2
  float rk[D + 1], su[D], sq[D];       // row k of A (and |x|^2), u and q: broadcast copies in the reduction
  float2 br[D];                        // brackets (lo, hi] of the eigenvalues, ascending order
  float x[NT];                         // multisection points of one pass
  int cnt[NT];                         // their Sturm counts
  float P[D][D];                       // inverse iteration: reciprocal LDL^T pivots, [i][eigenvalue]
  float bounds[2];                     // Gershgorin interval of T
  float scale;                         // max |A_ii|: the size of the matrix
};

// number of eigenvalues of T below x (the LDL^T pivots of T - x I that are
// negative); a pivot smaller than pivmin in magnitude is taken as -pivmin
template <int D>
__device__ __forceinline__ int sturm_count(const float* __restrict__ d, const float* __restrict__ e2, float x,
                                           float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int c = q < 0.f;
#pragma unroll
  for (int i = 1; i < D; ++i) {
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

// passes of the bracket multisection until every bracket is below 2^-24 of
// the first interval: (NT + 1) (per + 1)^passes >= 2^24
__host__ __device__ constexpr int multisection_passes(int nt, int per) {
  double w = double(nt + 1);
  int p = 0;
  while (w < 16777216.0 && p < 24) {
    w *= double(per + 1);
    ++p;
  }
  return p;
}

// Eigenvector estimates of the symmetric D x D matrix As (shared memory,
// row-major float32), written to V (column k belongs to the k-th smallest
// eigenvalue of the reduced matrix; row-major, stride D); mu[k] receives that
// eigenvalue (float32 resolution).  Run by threads 0..NT-1 of the block;
// `bar` synchronises exactly those threads.  D <= NT.
//
// The loops over the reduction steps, the multisection passes, the inverse
// iterations and the reflections run as loops: unrolled, their straight-line
// code (tens of thousands of instructions, each executed once) is fetched
// faster than it issues only from the instruction cache, which it overflows.
// The loops over matrix entries inside them are unrolled, so the rows and
// vectors stay in registers.
template <int D, int NT, typename Bar>
__device__ void eig_vectors_f32(const float* __restrict__ As, TridiagSmem<D, NT>& w, float* __restrict__ V,
                                float* __restrict__ mu, Bar bar) {
  static_assert(D >= 1 && D <= NT && D <= 64, "one warp reduces the matrix; one thread per eigenvalue");
  constexpr int R = (D + 31) / 32;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  constexpr unsigned kFull = 0xffffffffu;

  // ---- 1. Householder reduction.  D <= 32: every warp of the block holds
  // rows of A (row i in warp i mod W, lane j its column j), so each step's
  // products are warp reductions running side by side, with two barriers a
  // step; D > 32: warp 0 alone, a row of A a lane (two for D > 32).
  if constexpr (D <= 32) {
    constexpr int W = (NT / 32) < D ? (NT / 32) : D;  // warps holding rows
    constexpr int RPW = (D + W - 1) / W;              // rows a warp holds
    const int warp = tid >> 5;
    float a[RPW];
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const int row = warp + r * W;
      a[r] = (warp < W && row < D && lane < D) ? As[row * D + lane] : 0.f;
    }
    float scale = 0.f;
    for (int j = 0; j < D; ++j) scale = fmaxf(scale, fabsf(As[j * D + j]));
    const float skip = 1e-12f * scale;  // a column below this size is taken as already reduced
#pragma unroll 1
    for (int k = 0; k + 2 < D; ++k) {
      // the owner of row k (= column k below the diagonal, A being symmetric)
      // forms u = x - alpha e_1 with alpha = -sign(x_0) |x|, so |u|^2 = 2 h
      if (warp == k % W) {
        float ak = 0.f;
#pragma unroll
        for (int r = 0; r < RPW; ++r)
          if (r == k / W) ak = a[r];
        const float v = lane > k && lane < D ? ak : 0.f;
        float xs = v * v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) xs += __shfl_xor_sync(kFull, xs, o);
        const float x0 = __shfl_sync(kFull, v, k + 1);
        const float nx = sqrtf(xs);
        const bool reflect = nx > skip && xs > 0.f;  // warp-uniform
        const float alpha = x0 > 0.f ? -nx : nx;
        const float h = reflect ? fmaf(-x0, alpha, xs) : 0.f;
        const float u = !reflect ? 0.f : (lane == k + 1 ? x0 - alpha : v);
        if (lane < D) {
          w.U[k][lane] = u;
          w.su[lane] = u;
        }
        if (lane == 0) w.h[k] = h;
      }
      bar();
      const float h = w.h[k];
      if (!(h > 0.f)) continue;  // the same for every thread
      const float uj = lane < D ? w.su[lane] : 0.f;
      const float ih = __frcp_rn(h);
      // p_i = (A u)_i / h for this warp's rows
      float p[RPW];
#pragma unroll
      for (int r = 0; r < RPW; ++r) {
        float t = a[r] * uj;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
        p[r] = t * ih;
        const int row = warp + r * W;
        if (lane == 0 && warp < W && row < D) w.sq[row] = p[r];
      }
      bar();
      // K = u^T p / (2 h), q = p - K u, A <- A - u q^T - q u^T
      const float pj = lane < D ? w.sq[lane] : 0.f;
      float up = uj * pj;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) up += __shfl_xor_sync(kFull, up, o);
      const float K = 0.5f * up * ih;
      const float qj = fmaf(-K, uj, pj);
#pragma unroll
      for (int r = 0; r < RPW; ++r) {
        const int row = warp + r * W;
        const float ui = __shfl_sync(kFull, uj, row & 31);
        const float qi = fmaf(-K, ui, p[r]);
        a[r] = fmaf(-ui, qj, fmaf(-qi, uj, a[r]));
      }
    }
    // T: diagonal and first off-diagonal, from the owners of the rows
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const int row = warp + r * W;
      const float nxt = __shfl_down_sync(kFull, a[r], 1);  // the entry right of lane's
      if (warp < W && row < D && lane == row) {
        w.d[row] = a[r];
        if (row + 1 < D) {
          w.e[row] = nxt;
          w.e2[row] = nxt * nxt;
        }
      }
    }
    if (tid == 0) {
      w.e[D - 1] = 0.f;
      w.e2[D - 1] = 0.f;
      w.scale = scale;
    }
    bar();
  }
  if (tid < 32) {
    if constexpr (D > 32) {
      float a[R][D];
      float scale = 0.f;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int row = r * 32 + lane;
#pragma unroll
        for (int j = 0; j < D; ++j) a[r][j] = row < D ? As[row * D + j] : 0.f;
#pragma unroll
        for (int j = 0; j < D; ++j)
          if (row == j) scale = fmaxf(scale, fabsf(a[r][j]));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) scale = fmaxf(scale, __shfl_xor_sync(kFull, scale, o));
      const float skip = 1e-12f * scale;  // a column below this size is taken as already reduced
#pragma unroll 1
      for (int k = 0; k + 2 < D; ++k) {
        // column k of A, below the diagonal, read as row k (A is symmetric):
        // its owner lane publishes the row and |x|^2
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (r * 32 + lane == k) {
            float t0 = 0.f, t1 = 0.f;
#pragma unroll
            for (int j = 0; j < D; ++j) {
              w.rk[j] = a[r][j];
              const float v = j > k ? a[r][j] : 0.f;
              if (j & 1) t1 = fmaf(v, v, t1);
              else t0 = fmaf(v, v, t0);
            }
            w.rk[D] = t0 + t1;
          }
        }
        __syncwarp();
        float xv[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int row = r * 32 + lane;
          xv[r] = (row > k && row < D) ? w.rk[row] : 0.f;
        }
        const float xs = w.rk[D];
        const float x0 = w.rk[k + 1];
        const float nx = sqrtf(xs);
        const bool reflect = nx > skip && xs > 0.f;  // warp-uniform
        // u = x - alpha e_1 with alpha = -sign(x_0) |x|, so |u|^2 = 2 (|x|^2 + |x_0| |x|)
        const float alpha = x0 > 0.f ? -nx : nx;
        const float h = reflect ? fmaf(-x0, alpha, xs) : 0.f;
        float u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int row = r * 32 + lane;
          u[r] = !reflect ? 0.f : (row == k + 1 ? x0 - alpha : (row > k + 1 ? xv[r] : 0.f));
          if (row < D) {
            w.U[k][row] = u[r];
            w.su[row] = u[r];
          }
        }
        if (lane == 0) w.h[k] = h;
        __syncwarp();
        if (reflect) {
          // p = A u / h, K = u^T p / (2 h), q = p - K u, A <- A - u q^T - q u^T
          const float ih = __frcp_rn(h);
          float p[R];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int row = r * 32 + lane;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int j = 0; j < D; j += 3) {
              s0 = fmaf(a[r][j], w.su[j], s0);
              if (j + 1 < D) s1 = fmaf(a[r][j + 1], w.su[j + 1], s1);
              if (j + 2 < D) s2 = fmaf(a[r][j + 2], w.su[j + 2], s2);
            }
            p[r] = (s0 + s1 + s2) * ih;
            if (row < D) w.sq[row] = p[r];
          }
          __syncwarp();
          // u^T p, summed by every lane from the broadcast copies (no shuffle chain)
          float up0 = 0.f, up1 = 0.f, up2 = 0.f;
#pragma unroll
          for (int j = 0; j < D; j += 3) {
            up0 = fmaf(w.su[j], w.sq[j], up0);
            if (j + 1 < D) up1 = fmaf(w.su[j + 1], w.sq[j + 1], up1);
            if (j + 2 < D) up2 = fmaf(w.su[j + 2], w.sq[j + 2], up2);
          }
          const float up = up0 + up1 + up2;
          __syncwarp();
          const float K = 0.5f * up * ih;
          float q[R];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int row = r * 32 + lane;
            q[r] = fmaf(-K, u[r], p[r]);
            if (row < D) w.sq[row] = q[r];
          }
          __syncwarp();
#pragma unroll
          for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int j = 0; j < D; ++j) a[r][j] = fmaf(-u[r], w.sq[j], fmaf(-q[r], w.su[j], a[r][j]));
          }
        }
        __syncwarp();
      }
      // T: diagonal and first off-diagonal
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int row = r * 32 + lane;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          if (row == j) {
            w.d[j] = a[r][j];
            if (j + 1 < D) {
              w.e[j] = a[r][j + 1];
              w.e2[j] = a[r][j + 1] * a[r][j + 1];
            }
          }
        }
      }
      if (lane == 0) {
        w.e[D - 1] = 0.f;
        w.e2[D - 1] = 0.f;
        w.scale = scale;
      }
      __syncwarp();
    }
    // Gershgorin interval of T
    float glo = 3.0e38f, ghi = -3.0e38f;
    for (int i = lane; i < D; i += 32) {
      const float rad = fabsf(w.e[i]) + (i > 0 ? fabsf(w.e[i - 1]) : 0.f);
      glo = fminf(glo, w.d[i] - rad);
      ghi = fmaxf(ghi, w.d[i] + rad);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      glo = fminf(glo, __shfl_xor_sync(kFull, glo, o));
      ghi = fmaxf(ghi, __shfl_xor_sync(kFull, ghi, o));
    }
    const float pad = 1e-6f * fmaxf(fabsf(glo), fabsf(ghi)) + 1e-30f;
    if (lane == 0) {
      w.bounds[0] = glo - pad;
      w.bounds[1] = ghi + pad;
    }
    for (int i = lane; i < D; i += 32) w.br[i] = make_float2(glo - pad, ghi + pad);
  }
  bar();

  const float scale = w.scale;
  if (!(scale > 0.f)) {
    // the zero matrix: every eigenvalue is 0, any basis will do
    for (int i = tid; i < D * D; i += NT) V[i] = (i / D == i % D) ? 1.f : 0.f;
    for (int i = tid; i < D; i += NT) mu[i] = 0.f;
    bar();
    return;
  }
  float emax2 = 0.f;
#pragma unroll
  for (int i = 0; i + 1 < D; ++i) emax2 = fmaxf(emax2, w.e2[i]);
  const float pivmin = 1e-30f * fmaxf(1.f, emax2);

  // ---- 2. multisection.  Pass 0 counts at NT points across the whole
  // interval; a crossing between points t - 1 and t brackets the eigenvalues
  // k with cnt[t-1] <= k < cnt[t].  Later passes put kPer points in each
  // bracket.  (The counts do not decrease along x; if rounding ever made
  // them, an eigenvalue left without a new bracket keeps its old one.)
  {
    const float lo = w.bounds[0], hi = w.bounds[1];
    const float x = lo + (hi - lo) * (float(tid + 1) / float(NT + 1));
    w.x[tid] = x;
    w.cnt[tid] = sturm_count<D>(w.d, w.e2, x, pivmin);
  }
  bar();
  {
    const int c = w.cnt[tid];
    const int c0 = tid == 0 ? 0 : w.cnt[tid - 1];
    const float x0 = tid == 0 ? w.bounds[0] : w.x[tid - 1];
    for (int k = max(c0, 0); k < min(c, D); ++k) w.br[k] = make_float2(x0, w.x[tid]);
    if (tid == NT - 1)
      for (int k = max(c, 0); k < D; ++k) w.br[k] = make_float2(w.x[tid], w.bounds[1]);
  }
  bar();
  constexpr int kPer = TridiagSmem<D, NT>::kPer;
  constexpr int kPasses = multisection_passes(NT, kPer);
  const bool sect = tid < D * kPer;
  const int sk = tid / kPer, sj = tid % kPer;
#pragma unroll 1
  for (int pass = 0; pass < kPasses; ++pass) {
    float2 b = make_float2(0.f, 0.f);
    if (sect) {
      b = w.br[sk];
      const float x = b.x + (b.y - b.x) * (float(sj + 1) / float(kPer + 1));
      w.x[tid] = x;
      w.cnt[tid] = sturm_count<D>(w.d, w.e2, x, pivmin);
    }
    bar();
    if (sect) {
      // the first of the bracket's points whose count exceeds k sets the new
      // bracket; if none does, the last point and the old upper end
      const bool f = w.cnt[tid] > sk;
      const bool fp = sj > 0 && w.cnt[tid - 1] > sk;
      if (f && !fp) w.br[sk] = make_float2(sj == 0 ? b.x : w.x[tid - 1], w.x[tid]);
      else if (!f && sj == kPer - 1) w.br[sk] = make_float2(w.x[tid], b.y);
    }
    bar();
  }

  // ---- 3. inverse iteration, thread k for eigenvalue k; 4. back to A's basis
  if (tid < D) {
    const int k = tid;
    const float m = 0.5f * (w.br[k].x + w.br[k].y);
    mu[k] = m;
    const float tiny = scale * 5.9604645e-8f;  // 2^-24 of the matrix
    // LDL^T of T - m I, pivots guarded against tiny ones; P holds their
    // reciprocals (the same factors serve both iterations)
    {
      float piv = w.d[0] - m;
      if (fabsf(piv) < tiny) piv = piv < 0.f ? -tiny : tiny;
      float rp = __frcp_rn(piv);
      w.P[0][k] = rp;
#pragma unroll 4
      for (int i = 1; i < D; ++i) {
        piv = fmaf(-(w.e[i - 1] * rp), w.e[i - 1], w.d[i] - m);
        if (fabsf(piv) < tiny) piv = piv < 0.f ? -tiny : tiny;
        rp = __frcp_rn(piv);
        w.P[i][k] = rp;
      }
    }
    float z[D];
    // a start vector with no special direction: entries in [0.5, 1.5)
#pragma unroll
    for (int i = 0; i < D; ++i) {
      const float f = float(i) * 0.61803398875f + float(k) * 0.41421356237f;
      z[i] = 0.5f + (f - floorf(f));
    }
#pragma unroll 1
    for (int it = 0; it < 2; ++it) {
      // solve L D L^T y = z: forward with L (multipliers e_{i-1} / piv_{i-1}),
      // scale by D^-1, back with L^T
#pragma unroll
      for (int i = 1; i < D; ++i) z[i] = fmaf(-(w.e[i - 1] * w.P[i - 1][k]), z[i - 1], z[i]);
      z[D - 1] *= w.P[D - 1][k];
      float ymax = fabsf(z[D - 1]);
#pragma unroll
      for (int i = D - 2; i >= 0; --i) {
        const float rpi = w.P[i][k];
        z[i] = fmaf(-(w.e[i] * rpi), z[i + 1], z[i] * rpi);
        ymax = fmaxf(ymax, fabsf(z[i]));
      }
      // normalise (by the largest entry first, so the sum of squares cannot overflow)
      const float is = ymax > 0.f ? __frcp_rn(ymax) : 1.f;
      float ss = 0.f;
#pragma unroll
      for (int i = 0; i < D; ++i) {
        z[i] *= is;
        ss = fmaf(z[i], z[i], ss);
      }
      const float nrm = rsqrtf(ss);
#pragma unroll
      for (int i = 0; i < D; ++i) z[i] *= nrm;
    }
    // v = H_0 H_1 ... H_{D-3} z; u_s is zero in entries 0..s, so the
    // products run over all D entries
#pragma unroll 1
    for (int s = D - 3; s >= 0; --s) {
      const float hs = w.h[s];
      if (!(hs > 0.f)) continue;
      const float* us = w.U[s];
      float t0 = 0.f, t1 = 0.f, t2 = 0.f;
#pragma unroll
      for (int i = 0; i < D; i += 3) {
        t0 = fmaf(us[i], z[i], t0);
        if (i + 1 < D) t1 = fmaf(us[i + 1], z[i + 1], t1);
        if (i + 2 < D) t2 = fmaf(us[i + 2], z[i + 2], t2);
      }
      const float c = (t0 + t1 + t2) * __frcp_rn(hs);
#pragma unroll
      for (int i = 0; i < D; ++i) z[i] = fmaf(-c, us[i], z[i]);
    }
#pragma unroll
    for (int i = 0; i < D; ++i) V[i * D + k] = z[i];
  }
  bar();
}

}  // namespace
}  // namespace fgbd
