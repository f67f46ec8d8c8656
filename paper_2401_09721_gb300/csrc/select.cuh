// FSLR selection (Eq. 6, Section 2.4) and the graph low-pass filter (Eq. 5)
// as one device routine, run by the blocks of a cooperative grid: the
// selection kernel (k_filter) and, inside the noise-estimate launch, the
// blocks that took the first steps while sigma_est was computed.
//
//   phase 0   the FSLR keep flag of each point (spread <= 2 sigma_est) goes to
//             keep8; the kept power sum y^2 and the kept count are reduced, and
//             so are the stored steps' per-point power sums x_q^2;
//             x_0 = y is written unless steps are stored.
//   J(1..S)   from those sums, by thread 0 of every block (the same values
//             everywhere: the sums are exact integers).
//   step t    x_t = x_{t-1}/2 + (sum_j e_j x_{t-1}[j]) / (2 sum_j e_j) with
//             e_j = exp(-(d2_j - min_j d2_j) / sigma_g^2) (eq5_step): the rows
//             of D^{-1} W of Eq. 4, normalised once per graph by step 1 (from
//             the neighbours' coordinates, carried in x.w) and read back by the
//             later steps.
//             In select mode the kept power sum x_t^2 is reduced and, after a
//             grid barrier, J(t) = |sigma^2 - (sum y^2 - sum x_t^2)/(3 N_sel)|;
//             the search stops at the first t with J(t) >= J(t-1), keeping
//             q* = t-1.
//   output    the kept iterate is gathered back to input order (optional).
// Data written earlier in the same launch by other blocks (stored steps, the
// iterates, keep flags, sigma_est) is read through L2 only (ld.global.cg):
// the L1 caches of different SMs are not coherent within a grid.
// Sums of squares are fixed-point integers (2^-8), so the reduction is exact
// and independent of the order in which blocks add.  Grid barriers have a 2 s
// wait limit; a block that gives up latches kFlagTimeout and every block
// returns.
#pragma once

#include <climits>

#include "filter_step.cuh"

namespace fgbd {
namespace {

// ---- float-float arithmetic (an unevaluated sum hi + lo of two floats,
// about 44 significant bits): the error-free transformations TwoSum (Knuth)
// and TwoProduct through a fused multiply-add, as in Dekker's double-length
// arithmetic.  Float64 is slow on this GPU; this stands in for it in the rare
// FSLR decisions that float32 cannot take.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_add(FF x, FF y) {
  const float s = __fadd_rn(x.hi, y.hi);
  const float bb = __fsub_rn(s, x.hi);
  const float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));
  return ff_fast_two_sum(s, __fadd_rn(e, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ FF ff_neg(FF x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
  const float p = __fmul_rn(x.hi, y.hi);
  const float e = fmaf(x.hi, y.hi, -p);
  return ff_fast_two_sum(p, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e)));
}
__device__ __forceinline__ FF ff_div_int(FF x, int k) {
  const float kf = float(k);
  const float q1 = __fdiv_rn(x.hi, kf);
  const FF r = ff_add(x, ff_neg(ff_mul({q1, 0.f}, {kf, 0.f})));
  return ff_fast_two_sum(q1, __fdiv_rn(r.hi, kf));
}
__device__ __forceinline__ FF ff_sqrt(FF x) {
  if (!(x.hi > 0.f)) return {0.f, 0.f};
  const float s = __fsqrt_rn(x.hi);
  const FF r = ff_add(x, ff_neg(ff_mul({s, 0.f}, {s, 0.f})));
  return ff_fast_two_sum(s, __fdiv_rn(r.hi, __fmul_rn(2.f, s)));
}

// The FSLR keep decision of Section 2.4, spread <= threshold, for a point whose
// float32 spread is too close to the threshold to decide.  The spread is the
// mean of the three population standard deviations over the point and its
// neighbours; the decision compares their sum with 3 thr (thr as float-float).
// uint8 colours: cnt^2 times each variance is the integer cnt sum x^2 - (sum x)^2
// (below 2^22, exact in float32), so only the three square roots need float-float.
// float colours: two-pass (mean, then squared deviations) in float-float.
__device__ __noinline__ bool keep_ff(const FilterArgs& a, int k, FF thr) {
  int nb[7];
  bool v[7];
  const uint32_t pkk = a.pk[k];
  nb[0] = k;
  v[0] = true;
  nb[1] = k - 1;
  v[1] = c1_prev_linked(pkk, k);
  nb[2] = k + 1;
  v[2] = c1_next_linked(pkk, k, a.n);
  const int4 s = a.c4[k];
  nb[3] = s.x;
  nb[4] = s.y;
  nb[5] = s.z;
  nb[6] = s.w;
#pragma unroll
  for (int j = 3; j < 7; ++j) v[j] = in_range(nb[j], a.n);
  int cnt = 0;
#pragma unroll
  for (int j = 0; j < 7; ++j) cnt += v[j];
  FF total = {0.f, 0.f};
  if (a.dtype == 0) {
    uint32_t c[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) c[j] = v[j] ? a.y8[nb[j]] : 0u;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      int sx = 0, sq = 0;
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        const int x = int((c[j] >> (8 * ch)) & 255u);
        sx += x;
        sq += x * x;
      }
      const int V = cnt * sq - sx * sx;  // cnt^2 var; absent neighbours read as 0 and add nothing
      total = ff_add(total, ff_sqrt({float(V), 0.f}));
    }
    // sum_c sqrt(V_c) / cnt against 3 thr
    const FF d = ff_add(total, ff_neg(ff_mul(thr, {3.f * float(cnt), 0.f})));
    return d.hi < 0.f || (d.hi == 0.f && d.lo <= 0.f);
  }
  float col[3][7];
#pragma unroll
  for (int j = 0; j < 7; ++j) {
    if (v[j]) {
      const float4 y = a.yf[nb[j]];
      col[0][j] = y.x;
      col[1][j] = y.y;
      col[2][j] = y.z;
    } else {
      col[0][j] = col[1][j] = col[2][j] = 0.f;
    }
  }
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    FF sum = {0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 7; ++j)
      if (v[j]) sum = ff_add(sum, {col[ch][j], 0.f});
    const FF mean = ff_div_int(sum, cnt);
    FF ss = {0.f, 0.f};
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      if (v[j]) {
        const FF d = ff_add({col[ch][j], 0.f}, ff_neg(mean));
        ss = ff_add(ss, ff_mul(d, d));
      }
    }
    total = ff_add(total, ff_sqrt(ff_div_int(ss, cnt)));
  }
  const FF d = ff_add(total, ff_neg(ff_mul(thr, {3.f, 0.f})));
  return d.hi < 0.f || (d.hi == 0.f && d.lo <= 0.f);
}

// The same decision at a window w > 1: the point and its 6 + NX neighbour
// slots, in loops (only the few points in the float32 band come here).
template <int NX>
__device__ __noinline__ bool keep_ff_wide(const FilterArgs& a, int k, FF thr) {
  const int n = a.n;
  const uint32_t pkk = a.pk[k];
  const int4 s = a.c4[k];
  FF total = {0.f, 0.f};
  int cnt = 1;
#pragma unroll 1
  for (int j = 0; j < 6 + NX; ++j) cnt += neighbour_of(j, k, n, pkk, s, a.cx, a.cx_stride) >= 0;
  if (a.dtype == 0) {
    int sx[3], sq[3];
    const uint32_t own = a.y8[k];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const int x = int((own >> (8 * ch)) & 255u);
      sx[ch] = x;
      sq[ch] = x * x;
    }
#pragma unroll 1
    for (int j = 0; j < 6 + NX; ++j) {
      const int o = neighbour_of(j, k, n, pkk, s, a.cx, a.cx_stride);
      if (o < 0) continue;
      const uint32_t c = a.y8[o];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const int x = int((c >> (8 * ch)) & 255u);
        sx[ch] += x;
        sq[ch] += x * x;
      }
    }
    // cnt^2 var <= 19^2 127.5^2 < 2^24: exact in float32
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) total = ff_add(total, ff_sqrt({float(cnt * sq[ch] - sx[ch] * sx[ch]), 0.f}));
    const FF d = ff_add(total, ff_neg(ff_mul(thr, {3.f * float(cnt), 0.f})));
    return d.hi < 0.f || (d.hi == 0.f && d.lo <= 0.f);
  }
#pragma unroll 1
  for (int ch = 0; ch < 3; ++ch) {
    const float* own = reinterpret_cast<const float*>(&a.yf[k]);
    FF sum = {own[ch], 0.f};
#pragma unroll 1
    for (int j = 0; j < 6 + NX; ++j) {
      const int o = neighbour_of(j, k, n, pkk, s, a.cx, a.cx_stride);
      if (o >= 0) sum = ff_add(sum, {reinterpret_cast<const float*>(&a.yf[o])[ch], 0.f});
    }
    const FF mean = ff_div_int(sum, cnt);
    FF dd = ff_add({own[ch], 0.f}, ff_neg(mean));
    FF ss = ff_mul(dd, dd);
#pragma unroll 1
    for (int j = 0; j < 6 + NX; ++j) {
      const int o = neighbour_of(j, k, n, pkk, s, a.cx, a.cx_stride);
      if (o < 0) continue;
      dd = ff_add({reinterpret_cast<const float*>(&a.yf[o])[ch], 0.f}, ff_neg(mean));
      ss = ff_add(ss, ff_mul(dd, dd));
    }
    total = ff_add(total, ff_sqrt(ff_div_int(ss, cnt)));
  }
  const FF d = ff_add(total, ff_neg(ff_mul(thr, {3.f, 0.f})));
  return d.hi < 0.f || (d.hi == 0.f && d.lo <= 0.f);
}

template <int NX>
__device__ __forceinline__ bool keep_ff_nx(const FilterArgs& a, int k, FF thr) {
  if constexpr (NX == 0) return keep_ff(a, k, thr);
  else return keep_ff_wide<NX>(a, k, thr);
}

__device__ __forceinline__ void write_out(const FilterArgs& a, int i, float4 x) {
  if (a.out_dtype == 0) {
    uint8_t* o = static_cast<uint8_t*>(a.out) + 3 * size_t(i);
    o[0] = uint8_t(fminf(fmaxf(rintf(x.x), 0.f), 255.f));
    o[1] = uint8_t(fminf(fmaxf(rintf(x.y), 0.f), 255.f));
    o[2] = uint8_t(fminf(fmaxf(rintf(x.z), 0.f), 255.f));
  } else {
    float* o = static_cast<float*>(a.out) + 3 * size_t(i);
    o[0] = x.x;
    o[1] = x.y;
    o[2] = x.z;
  }
}

// x_q of sorted point k, wherever the kept iterate is (kept_buf)
__device__ __forceinline__ float4 kept_value(const FilterArgs& a, int kept, int k) {
  if (kept < 0) return x0_of(a, k);
  if (kept == kKeptBest) return __ldcg(&a.xbest[k]);
  if (kept >= 2) return __ldcg(&a.spec_x[size_t(kept - 2) * size_t(a.cap) + k]);
  return __ldcg(&(kept ? a.xbuf1 : a.xbuf0)[k]);
}

// x_0 of the sorted points k0 .. k0 + 3 (k0 a multiple of 4; those at or past
// n only when `full` is false, and then left unread).  The packed coordinates
// (x.w) are read only when `with_pk`.
__device__ __forceinline__ void x0_quad(const FilterArgs& a, int k0, bool full, bool with_pk, float4 (&x)[4]) {
  uint32_t p[4] = {0u, 0u, 0u, 0u};
  if (with_pk) {
    if (full) {
      const uint4 v = *reinterpret_cast<const uint4*>(a.pk + k0);
      p[0] = v.x;
      p[1] = v.y;
      p[2] = v.z;
      p[3] = v.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (k0 + i < a.n) p[i] = a.pk[k0 + i];
    }
  }
  if (a.dtype == 0) {
    uint32_t y[4] = {0u, 0u, 0u, 0u};
    if (full) {
      const uint4 v = *reinterpret_cast<const uint4*>(a.y8 + k0);
      y[0] = v.x;
      y[1] = v.y;
      y[2] = v.z;
      y[3] = v.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (k0 + i < a.n) y[i] = a.y8[k0 + i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      x[i] = make_float4(float(y[i] & 255u), float((y[i] >> 8) & 255u), float((y[i] >> 16) & 255u),
                         __uint_as_float(p[i]));
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 c = (full || k0 + i < a.n) ? a.yf[k0 + i] : make_float4(0.f, 0.f, 0.f, 0.f);
      x[i] = make_float4(c.x, c.y, c.z, __uint_as_float(p[i]));
    }
  }
}

// colours of the kept iterate at sorted point k (x.w is not meaningful)
__device__ __forceinline__ float4 kept_rgb(const FilterArgs& a, int kept, int k) {
  if (kept < 0) {
    float r, g, b;
    load_y(a, k, r, g, b);
    return make_float4(r, g, b, 0.f);
  }
  return kept_value(a, kept, k);
}

// The kept iterate in input order: input points i0 .. i0 + 3 per thread and
// trip, their sorted positions read as one int4 and the four gathers issued
// together; uint8 / float32 output as 32- / 128-bit stores where aligned.
__device__ __forceinline__ void output_quads(const FilterArgs& a, int kept, int gtid, int gstride) {
  const int n = a.n;
  const bool u8 = a.out_dtype == 0;
  const bool wide = (reinterpret_cast<uintptr_t>(a.out) & (u8 ? 3u : 15u)) == 0;
  for (int i0 = 4 * gtid; i0 < n; i0 += 4 * gstride) {
    const bool full = i0 + 4 <= n;
    int kk[4] = {-1, -1, -1, -1};
    if (full) {
      const int4 v = *reinterpret_cast<const int4*>(a.rank1 + i0);
      kk[0] = v.x;
      kk[1] = v.y;
      kk[2] = v.z;
      kk[3] = v.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (i0 + i < n) kk[i] = a.rank1[i0 + i];
    }
    float4 v[4];
    bool ok[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      ok[i] = in_range(kk[i], n);
      v[i] = ok[i] ? kept_rgb(a, kept, kk[i]) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (full && wide && ok[0] && ok[1] && ok[2] && ok[3]) {
      if (u8) {
        uint32_t b[12];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          b[3 * i + 0] = uint32_t(fminf(fmaxf(rintf(v[i].x), 0.f), 255.f));
          b[3 * i + 1] = uint32_t(fminf(fmaxf(rintf(v[i].y), 0.f), 255.f));
          b[3 * i + 2] = uint32_t(fminf(fmaxf(rintf(v[i].z), 0.f), 255.f));
        }
        uint32_t* o = reinterpret_cast<uint32_t*>(static_cast<uint8_t*>(a.out) + 3 * size_t(i0));
#pragma unroll
        for (int w = 0; w < 3; ++w)
          o[w] = b[4 * w] | (b[4 * w + 1] << 8) | (b[4 * w + 2] << 16) | (b[4 * w + 3] << 24);
      } else {
        float4* o = reinterpret_cast<float4*>(static_cast<float*>(a.out) + 3 * size_t(i0));
        o[0] = make_float4(v[0].x, v[0].y, v[0].z, v[1].x);
        o[1] = make_float4(v[1].y, v[1].z, v[2].x, v[2].y);
        o[2] = make_float4(v[2].z, v[3].x, v[3].y, v[3].z);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (ok[i] && i0 + i < n) write_out(a, i0 + i, v[i]);
    }
  }
}

// Sums of several 64-bit values over the block (two's complement: exact in any order)
template <int K, int THREADS>
__device__ __forceinline__ void block_sums(unsigned long long (&v)[K], unsigned long long* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < K; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < K; ++i) s_red[i * (THREADS / 32) + warp] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < K) {
    unsigned long long t = 0;
    for (int w = 0; w < THREADS / 32; ++w) t += s_red[threadIdx.x * (THREADS / 32) + w];
    s_red[K * (THREADS / 32) + threadIdx.x] = t;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < K; ++i) v[i] = s_red[K * (THREADS / 32) + i];
  __syncthreads();
}

constexpr int kSums = 3 + 2 * kSpecMax;  // kept y^2, all y^2, kept count, then per stored step kept and all x_q^2

// The selection and filter for the blocks [first, first + members) of a
// cooperative grid of THREADS-thread blocks, from S stored steps (0: none),
// grid barriers on *bar (epoch: the barriers this grid has passed on it);
// NX further neighbour slots per point (window w > 1: NX = 6 (w - 1)).
template <int THREADS, int NX = 0>
__device__ __forceinline__ void select_filter(const FilterArgs& a, int S, int first, uint32_t members,
                                              uint32_t* bar, uint32_t& epoch) {
  __shared__ unsigned long long s_red[(kSums + 1) * (THREADS / 32)];
  __shared__ int s_ok;
  const int n = a.n;
  const int gtid = (int(blockIdx.x) - first) * THREADS + int(threadIdx.x);
  const int gstride = int(members) * THREADS;
  DevScalars* sc = a.sc;
  const bool select = a.mode == 0;
  // Block-uniform scalars, computed by thread 0: the FSLR threshold 2 sigma_est
  // as a float32 band [t_lo, t_hi] (outside it float32 decides) and as float-float.
  __shared__ float s_thr[4];
  if (threadIdx.x == 0 && select) {
    if (a.sigma_src == &sc->sigma_est && sc->fslr_ready) {
      // as the eigen step formed them with sigma_est (fslr_band, the same arithmetic)
#pragma unroll
      for (int i = 0; i < 4; ++i) s_thr[i] = sc->fslr_thr[i];
    } else {
      fslr_band(a.fslr_factor, __ldcg(a.sigma_src), a.dtype, s_thr);
    }
  }
  __syncthreads();
  float t_lo = 0.f, t_hi = 0.f;
  FF thr = {0.f, 0.f};
  if (select) {
    t_lo = s_thr[0];
    t_hi = s_thr[1];
    thr = {s_thr[2], s_thr[3]};
  }

  // ---- phase 0: keep flags and the Eq. 6 sums; x_0 = y unless the steps are stored.
  // Four consecutive points per thread and trip, read with 16-byte loads that
  // are all issued before the first is used.
  unsigned long long acc[kSums] = {};
  for (int k0 = 4 * gtid; k0 < n; k0 += 4 * gstride) {
    const bool full = k0 + 4 <= n;
    float4 x[4];
    x0_quad(a, k0, full, !S, x);
    float sp[4] = {0.f, 0.f, 0.f, 0.f};
    if (select) {
      if (full) {
        const float4 v = *reinterpret_cast<const float4*>(a.spread + k0);
        sp[0] = v.x;
        sp[1] = v.y;
        sp[2] = v.z;
        sp[3] = v.w;
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (k0 + i < n) sp[i] = a.spread[k0 + i];
      }
    }
    if (!S) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (full || k0 + i < n) a.xbuf0[k0 + i] = x[i];
    }
    if (select) {
      uint32_t kw = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (!full && k0 + i >= n) continue;
        bool keep;
        if (a.all_points || sp[i] <= t_lo) keep = true;
        else if (sp[i] > t_hi) keep = false;
        else keep = keep_ff_nx<NX>(a, k0 + i, thr);
        kw |= uint32_t(keep) << (8 * i);
        const unsigned long long q2 = sq3(x[i]);
        acc[1] += q2;
        if (keep) {
          acc[0] += q2;
          acc[2] += 1;
        }
      }
      if (full) {
        *reinterpret_cast<uint32_t*>(a.keep8 + k0) = kw;
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (k0 + i < n) a.keep8[k0 + i] = uint8_t((kw >> (8 * i)) & 1u);
      }
    }
  }
  // the stored steps' power sums (a second pass over this thread's own points and keep flags)
  if (S > 0) {
    for (int k0 = 4 * gtid; k0 < n; k0 += 4 * gstride) {
      const bool full = k0 + 4 <= n;
      uint32_t kw = 0;
      int32_t z[kSpecMax][4] = {};
      if (full) kw = *reinterpret_cast<const uint32_t*>(a.keep8 + k0);
#pragma unroll
      for (int q = 0; q < kSpecMax; ++q) {
        if (q < S) {
          const int32_t* zr = a.spec_z + size_t(q) * size_t(a.cap) + k0;
          if (full) {
            const int4 v = __ldcg(reinterpret_cast<const int4*>(zr));
            z[q][0] = v.x;
            z[q][1] = v.y;
            z[q][2] = v.z;
            z[q][3] = v.w;
          } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (k0 + i < n) z[q][i] = __ldcg(zr + i);
          }
        }
      }
      if (!full) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (k0 + i < n) kw |= uint32_t(a.keep8[k0 + i] != 0) << (8 * i);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const bool keep = (kw >> (8 * i)) & 1u;
#pragma unroll
        for (int q = 0; q < kSpecMax; ++q) {
          if (q < S) {
            const unsigned long long zz = (unsigned long long)(long long)z[q][i];
            acc[4 + 2 * q] += zz;
            if (keep) acc[3 + 2 * q] += zz;
          }
        }
      }
    }
  }
  if (select) {
    block_sums<kSums, THREADS>(acc, s_red);
    if (threadIdx.x == 0) {
      if (acc[0]) atomicAdd(&sc->ysq_keep, acc[0]);
      if (acc[1]) atomicAdd(&sc->ysq_all, acc[1]);
      if (acc[2]) atomicAdd(&sc->n_keep, acc[2]);
#pragma unroll
      for (int q = 0; q < kSpecMax; ++q) {
        if (q < S) {
          atomicAdd(reinterpret_cast<unsigned long long*>(&sc->spec_keep[q + 1]), acc[3 + 2 * q]);
          atomicAdd(reinterpret_cast<unsigned long long*>(&sc->spec_all[q + 1]), acc[4 + 2 * q]);
        }
      }
    }
  }
  if (!grid_barrier(bar, &sc->status, members, epoch, &s_ok, sc)) return;

  // J(0..S) from the stored terms, by thread 0 of each block (every block
  // reaches the same values: the sums are exact integers).  Under the global
  // reading (a.q_global) the search never stops early and q* is the argmin of
  // J over 0..q_max (the smaller q among equal values); a new best iterate
  // beyond the stored steps is copied to xbest while the next step reads it.
  __shared__ int s_ctl[6];  // keep_all, q_limit, q_final, stop, q_best, copy the last iterate
  __shared__ float s_cexp;
  const bool global = select && a.q_global;
  double sigma = 0.0, nsel = 1.0, J_prev = 0.0, J_best = 0.0;  // thread 0 only
  // J(t) = |sigma^2 - lost_t / (3 N_sel)| with lost_t the exact fixed-point sum of
  // y^2 - x_t^2: sigma^2 and 2^-kSqShift / (3 N_sel) are formed once, so each J
  // is one fused multiply-add (float64 operations have a long latency here)
  double sig2 = 0.0, inv3n = 0.0;  // thread 0 only
  int q_best = 0;                                               // thread 0 only
  unsigned long long ysq = 0;
  if (threadIdx.x == 0) {
    // every scalar this thread reads, loaded together (one round trip to L2)
    const uint32_t c_ready = sc->cexp_ready;
    const float c_val = sc->cexp;
    unsigned long long nkt = 0, ysk = 0, ysa = 0, sk[kSpecMax] = {}, sa[kSpecMax] = {};
    if (select) {
      sigma = __ldcg(a.sigma_src);
      nkt = ld_relaxed_u64(&sc->n_keep);
      ysk = ld_relaxed_u64(&sc->ysq_keep);
      ysa = ld_relaxed_u64(&sc->ysq_all);
#pragma unroll
      for (int q = 0; q < kSpecMax; ++q) {
        if (q < S) {
          sk[q] = ld_relaxed_u64(reinterpret_cast<const unsigned long long*>(&sc->spec_keep[q + 1]));
          sa[q] = ld_relaxed_u64(reinterpret_cast<const unsigned long long*>(&sc->spec_all[q + 1]));
        }
      }
    }
    s_cexp = c_ready ? c_val : step_cexp(sc);
    const int q_fixed = a.q_src ? min(max(*a.q_src, 0), kQCap) : a.q_fixed;
    const int q_limit = n == 0 ? 0 : (select ? a.q_max : q_fixed);
    int keep_all = 0, q_final = 0, stopped = 0;
    if (select) {
      keep_all = nkt == 0;  // no point left: every point is used
      nsel = keep_all ? double(n) : double(nkt);
      ysq = keep_all ? ysa : ysk;
      sig2 = sigma * sigma;
      inv3n = (1.0 / double(1 << kSqShift)) / (3.0 * nsel);
      J_prev = sig2;  // J(0): nothing filtered yet
      J_best = J_prev;
      if (gtid == 0) sc->J[0] = J_prev;
#pragma unroll
      for (int t = 1; t <= kSpecMax; ++t) {
        if (t > min(S, q_limit)) break;
        // sum of y^2 - x_t^2 over the points of Eq. 6: exact in two's complement
        const double lost = double((long long)(ysq - (keep_all ? sa[t - 1] : sk[t - 1])));
        const double J = fabs(fma(-lost, inv3n, sig2));
        if (gtid == 0) {
          sc->J[t] = J;
          sc->n_J = t + 1;
        }
        if (global) {
          if (J < J_best) {
            J_best = J;
            q_best = t;
          }
          q_final = t;
          continue;
        }
        if (J >= J_prev) {
          q_final = t - 1;
          stopped = 1;
          break;
        }
        J_prev = J;
        q_final = t;
      }
    }
    s_ctl[0] = keep_all;
    s_ctl[1] = q_limit;
    s_ctl[2] = q_final;
    s_ctl[3] = stopped;
    s_ctl[4] = q_best;
    s_ctl[5] = 0;
  }
  __syncthreads();
  const float cexp = s_cexp;
  const bool keep_all = s_ctl[0] != 0;
  const int q_limit = s_ctl[1];
  int q_final = s_ctl[2];
  const bool stopped = s_ctl[3] != 0;
  bool copy_best = false;  // this step's source is the best iterate so far: copy it to xbest
  for (int t = S + 1; t <= q_limit && !stopped; ++t) {
    const float4* __restrict__ src =
        (S > 0 && t == S + 1) ? a.spec_x + size_t(S - 1) * size_t(a.cap) : ((t & 1) ? a.xbuf0 : a.xbuf1);
    float4* __restrict__ dst = (t & 1) ? a.xbuf1 : a.xbuf0;
    unsigned long long loc = 0;
    for (int k = gtid; k < n; k += gstride) {
      const StepHead h = step_head(a, src, k);
      const float4 xo =
          t == 1 ? eq5_step_nx<NX, true>(a, src, k, n, cexp, h) : eq5_step_nx<NX, false>(a, src, k, n, cexp, h);
      dst[k] = xo;
      if (copy_best) a.xbest[k] = h.xk;
      if (select && (keep_all || __ldcg(a.keep8 + k))) loc += sq3(xo);
    }
    if (select) {
      loc = block_sum_u64<THREADS>(loc, s_red);
      if (threadIdx.x == 0 && loc) atomicAdd(&sc->sumsq[t], loc);
    }
    // (the barrier starts with __syncthreads: every thread has read s_ctl[3])
    if (!grid_barrier(bar, &sc->status, members, epoch, &s_ok, sc)) return;
    if (select) {
      if (threadIdx.x == 0) {
        const unsigned long long ss = ld_relaxed_u64(&sc->sumsq[t]);
        const double lost = double((long long)(ysq - ss));
        const double J = fabs(fma(-lost, inv3n, sig2));
        if (gtid == 0) {
          sc->J[t] = J;
          sc->n_J = t + 1;
        }
        if (global) {
          const bool better = J < J_best;
          if (better) {
            J_best = J;
            q_best = t;
          }
          s_ctl[3] = 0;
          s_ctl[4] = q_best;
          s_ctl[5] = better;
        } else {
          s_ctl[3] = J >= J_prev;
          if (!(J >= J_prev)) J_prev = J;
        }
      }
      __syncthreads();
      if (s_ctl[3]) {
        q_final = t - 1;
        break;
      }
      q_final = t;
      copy_best = s_ctl[5] != 0;
    } else {
      q_final = t;
    }
  }
  // where the kept iterate is
  int kept = (S > 0 && q_final <= S) ? (q_final == 0 ? -1 : 2 + q_final - 1) : (q_final & 1);
  if (global) {
    const int qb = s_ctl[4];
    if (qb == 0) kept = -1;
    else if (qb <= S) kept = 2 + qb - 1;
    else if (qb == q_final) kept = qb & 1;  // the last step: still in its buffer
    else kept = kKeptBest;                  // copied while step qb + 1 read it
    q_final = qb;
  }
  if (gtid == 0) {
    if (!a.q_src) sc->q_sel = q_final;
    sc->kept_buf = kept;
    if (select) sc->sel_valid = 1;
    if (select && q_limit == 0) sc->n_J = 1;
  }
  if (a.out) output_quads(a, kept, gtid, gstride);
}

}  // namespace
}  // namespace fgbd
