// One step of the graph low-pass filter (Eq. 5) and the pieces around it that
// more than one kernel needs: the colours of the sorted points, the bounded
// grid barrier of the cooperative kernels, and the speculative steps that the
// noise-estimate kernel takes while its first block computes sigma_est.
#pragma once

#include <climits>

#include "fgbd_internal.cuh"

namespace fgbd {

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Barrier over `members` blocks of a cooperative grid: a counter that each
// block raises once per barrier, waited on for at most sc->wait_limit_ns (2 s
// unless a test lowers it); a block that gives up latches kFlagTimeout, and
// every block then returns false.
__device__ __forceinline__ bool grid_barrier(uint32_t* counter, uint32_t* status, uint32_t members, uint32_t& epoch,
                                             int* s_ok, const DevScalars* sc) {
  __syncthreads();
  epoch += 1;
  if (threadIdx.x == 0) {
    const uint32_t target = epoch * members;
    __threadfence();
    atomicAdd(counter, 1u);
    const unsigned long long t0 = global_ns();
    const unsigned long long limit = sc->wait_limit_ns;
    int ok = 1;
    while (ld_acquire_u32(counter) < target) {
      if (global_ns() - t0 > limit) {
        atomicOr(status, kFlagTimeout);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    if (ld_acquire_u32(status) & kFlagTimeout) ok = 0;
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

__device__ __forceinline__ void load_y(const FilterArgs& a, int k, float& r, float& g, float& b) {
  if (a.dtype == 0) {
    const uint32_t y = a.y8[k];
    r = float(y & 255u);
    g = float((y >> 8) & 255u);
    b = float((y >> 16) & 255u);
  } else {
    const float4 y = a.yf[k];
    r = y.x;
    g = y.y;
    b = y.z;
  }
}

// x_0 of sorted point k: its colour, and its packed coordinates in w
__device__ __forceinline__ float4 x0_of(const FilterArgs& a, int k) {
  float r, g, b;
  load_y(a, k, r, g, b);
  return make_float4(r, g, b, __uint_as_float(a.pk[k]));
}

// sum over the channels of x^2 in fixed point 2^-kSqShift
__device__ __forceinline__ unsigned long long sq3(float4 x) {
  return (unsigned long long)(sq_fixed(x.x) + sq_fixed(x.y) + sq_fixed(x.z));
}

// The FSLR threshold factor * sigma as the selection uses it: a float32 band
// [t[0], t[1]] outside which float32 decides, and the threshold as a
// float-float pair (t[2], t[3]).
__device__ __forceinline__ void fslr_band(double factor, double sigma, int dtype, float* t) {
  const double thr = factor * sigma;
  const double band = dtype == 0 ? 2e-6 : 5e-5;
  t[0] = float(thr * (1.0 - band));
  t[1] = float(thr * (1.0 + band));
  t[2] = float(thr);
  t[3] = float(thr - double(t[2]));
}

// The Eq. 4 exponent scale log2(e) / sigma_g^2
__device__ __forceinline__ float step_cexp(const DevScalars* sc) {
  const double sg = sigma_g_of(sc);
  return sg > 0.0 ? float(1.4426950408889634 / (sg * sg)) : 0.f;
}

// The same as the moments launch left it for this graph, or computed here:
// float64 work is slow on this GPU (dependent float64 operations cost hundreds
// of cycles), so it is done once where it is off the critical path.
__device__ __forceinline__ float graph_cexp(const DevScalars* sc) {
  return sc->cexp_ready ? sc->cexp : step_cexp(sc);
}

// The same, read or computed once per block by thread 0 and shared.
__device__ __forceinline__ float block_cexp(const DevScalars* sc, float* s_cexp) {
  if (threadIdx.x == 0) *s_cexp = graph_cexp(sc);
  __syncthreads();
  return *s_cexp;
}

// What a step at sorted point k reads before its neighbours: the point's own
// previous iterate (x_0 built from the colours when src is null) and its C2/C3
// slots.
struct StepHead {
  float4 xk;
  int4 s;
};

// An iterate of an earlier step: through L1 (kL1) where every line this SM
// could hold was final before the launch first read it - the stored steps of
// the noise-estimate launch, each writing a slice of its own that is only read
// after the next grid barrier - else from L2 (ping-pong buffers rewritten
// within one launch, whose stale L1 lines another SM could still hold).
template <bool kL1>
__device__ __forceinline__ float4 ld_iterate(const float4* __restrict__ p) {
  if constexpr (kL1) return __ldca(p);
  else return __ldcg(p);
}

template <bool kL1 = false>
__device__ __forceinline__ StepHead step_head(const FilterArgs& a, const float4* __restrict__ src, int k) {
  return {src ? ld_iterate<kL1>(&src[k]) : x0_of(a, k), a.c4[k]};
}

// The six window-1 slots of sorted point k (C1 k - 1, k + 1, then the C2/C3
// slots of c4) and whether each holds a neighbour.
__device__ __forceinline__ void slots6(int k, int n, uint32_t wk, int4 s, int (&nb)[6], bool (&v)[6]) {
  nb[0] = k - 1;
  v[0] = c1_prev_linked(wk, k);
  nb[1] = k + 1;
  v[1] = c1_next_linked(wk, k, n);
  nb[2] = s.x;
  nb[3] = s.y;
  nb[4] = s.z;
  nb[5] = s.w;
  v[2] = in_range(s.x, n);
  v[3] = in_range(s.y, n);
  v[4] = in_range(s.z, n);
  v[5] = in_range(s.w, n);
}

// One Eq. 5 step at sorted point k: x_k / 2 + (sum_j w_j x_j) / 2 over the
// neighbours (C1 k - 1, k + 1, the C2/C3 slots), with the weights of Eq. 4
// normalised by their sum, w_j = e_j / sum_i e_i, e_j = exp(-(d2_j - min d2) /
// sigma_g^2) (the pair reading: d2_j / (sigma_k sigma_j) in the exponent), from
// the previous iterate `src` (x_0 built from the colours when src is null;
// h = step_head(a, src, k)).  A point without neighbours keeps x_k.
// The weights depend on the graph and sigma_g only, so they are computed once:
// kStore (step 1) computes them and, where a.w4 is set, stores them; the later
// steps of the same graph load them (kStore false with a.w4 set).  Every kernel
// that takes a window-1 step uses this function, so a step gives the same bits
// in all of them.
template <bool kStore, bool kL1 = false>
__device__ __forceinline__ float4 eq5_step(const FilterArgs& a, const float4* __restrict__ src, int k, int n,
                                           float cexp, const StepHead& h) {
  const float4 xk = h.xk;
  const uint32_t wk = __float_as_uint(xk.w);  // packed code and the missing-C1-link bits
  int nb[6];
  bool v[6];
  slots6(k, n, wk, h.s, nb, v);
  float4 xn[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) xn[j] = v[j] ? (src ? ld_iterate<kL1>(&src[nb[j]]) : x0_of(a, nb[j])) : xk;
  float w[6];
  if (kStore || !a.w4) {
    const uint32_t ck = wk & kCoordMask;
    int d2[6];
    int dmin = INT_MAX;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      d2[j] = v[j] ? sq_dist_c1(ck, __float_as_uint(xn[j].w) & kCoordMask, a.bits) : INT_MAX;
      dmin = min(dmin, d2[j]);
    }
    float se = 0.f;
    if (a.node_sig) {
      // the pair reading: exponents d2_j / (sigma_k sigma_j), shifted by their minimum
      const float sk = __ldg(&a.node_sig[k]);
      float ex[6];
      float emin = 3.0e38f;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        ex[j] = 0.f;
        if (v[j]) {
          const float s = sk * __ldg(&a.node_sig[nb[j]]);
          ex[j] = s > 0.f ? float(d2[j]) / s : 0.f;
          emin = fminf(emin, ex[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        w[j] = v[j] ? exp2f((emin - ex[j]) * 1.4426950408889634f) : 0.f;
        se += w[j];
      }
    } else {
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        w[j] = v[j] ? exp2f(float(dmin - d2[j]) * cexp) : 0.f;
        se += w[j];
      }
    }
    // se >= 1 when a slot is linked (its nearest neighbour has e = 1)
    const float inv = se > 0.f ? 1.f / se : 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) w[j] *= inv;
    if (kStore && a.w4) {
      a.w4[k] = make_float4(w[0], w[1], w[2], w[3]);
      a.w2[k] = make_float2(w[4], w[5]);
    }
  } else {
    const float4 wa = __ldcg(&a.w4[k]);
    const float2 wb = __ldcg(&a.w2[k]);
    w[0] = wa.x;
    w[1] = wa.y;
    w[2] = wa.z;
    w[3] = wa.w;
    w[4] = wb.x;
    w[5] = wb.y;
  }
  float sr = 0.f, sgc = 0.f, sb = 0.f;
  bool any = false;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    if (v[j]) {
      sr = fmaf(w[j], xn[j].x, sr);
      sgc = fmaf(w[j], xn[j].y, sgc);
      sb = fmaf(w[j], xn[j].z, sb);
      any = true;
    }
  }
  float4 xo = xk;
  if (any) {
    xo.x = 0.5f * xk.x + 0.5f * sr;
    xo.y = 0.5f * xk.y + 0.5f * sgc;
    xo.z = 0.5f * xk.z + 0.5f * sb;
  }
  return xo;
}

// Slot group g of sorted point k as sorted ids (-1 empty): g = 0 the six
// window-1 slots (C1 k - 1, k + 1, the c4 slots), g >= 1 the further slots
// 6 (g - 1) .. 6 (g - 1) + 5 of a window w > 1.
__device__ __forceinline__ void slot_group(const FilterArgs& a, int k, int n, uint32_t wk, int4 s, int g, int (&o)[6]) {
  if (g == 0) {
#pragma unroll
    for (int i = 0; i < 6; ++i) o[i] = neighbour_of(i, k, n, wk, s, nullptr, 0);
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const int v = a.cx[size_t(6 * (g - 1) + i) * size_t(a.cx_stride) + k];
      o[i] = in_range(v, n) ? v : -1;
    }
  }
}

// The same step at a window w > 1, over the 6 + NX neighbours (NX = 6 (w - 1)
// further slots), six at a time so that the loads of a group are issued
// together: a first pass finds min d2 from the packed codes, a second
// accumulates.
template <int NX>
__device__ __forceinline__ float4 eq5_step_wide(const FilterArgs& a, const float4* __restrict__ src, int k, int n,
                                                float cexp, const StepHead& h) {
  const float4 xk = h.xk;
  const uint32_t wk = __float_as_uint(xk.w);
  const uint32_t ck = wk & kCoordMask;
  const int4 s = h.s;
  int dmin = INT_MAX;
#pragma unroll 1
  for (int g = 0; g <= NX / 6; ++g) {
    int o[6];
    slot_group(a, k, n, wk, s, g, o);
    uint32_t c[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) c[i] = o[i] >= 0 ? a.pk[o[i]] : 0u;
#pragma unroll
    for (int i = 0; i < 6; ++i)
      if (o[i] >= 0) dmin = min(dmin, sq_dist_c1(ck, c[i] & kCoordMask, a.bits));
  }
  float se = 0.f, sr = 0.f, sgc = 0.f, sb = 0.f;
#pragma unroll 1
  for (int g = 0; g <= NX / 6; ++g) {
    int o[6];
    slot_group(a, k, n, wk, s, g, o);
    float4 xo[6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
      xo[i] = o[i] >= 0 ? (src ? __ldcg(&src[o[i]]) : x0_of(a, o[i])) : xk;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      if (o[i] < 0) continue;
      const int d2 = sq_dist_c1(ck, __float_as_uint(xo[i].w) & kCoordMask, a.bits);
      const float e = exp2f(float(dmin - d2) * cexp);
      se += e;
      sr = fmaf(e, xo[i].x, sr);
      sgc = fmaf(e, xo[i].y, sgc);
      sb = fmaf(e, xo[i].z, sb);
    }
  }
  float4 xo = xk;
  if (se > 0.f) {
    const float inv = 1.f / se;
    xo.x = 0.5f * xk.x + 0.5f * (sr * inv);
    xo.y = 0.5f * xk.y + 0.5f * (sgc * inv);
    xo.z = 0.5f * xk.z + 0.5f * (sb * inv);
  }
  return xo;
}

// one Eq. 5 step at window 1 (NX = 0) or wider
template <int NX, bool kStore>
__device__ __forceinline__ float4 eq5_step_nx(const FilterArgs& a, const float4* __restrict__ src, int k, int n,
                                              float cexp, const StepHead& h) {
  if constexpr (NX == 0) return eq5_step<kStore>(a, src, k, n, cexp, h);
  else return eq5_step_wide<NX>(a, src, k, n, cexp, h);
}

// The first steps x_1, x_2, ... and beside them each point's sum_c x_q^2 in
// fixed point (the selection subtracts these sums from those of y^2 for
// Eq. 6), by the blocks [first, first + members) of a
// cooperative grid (they need the graph and the colours only, not sigma_est):
// `depth` steps, or, with `until_sigma`, fewer once sigma_est is published
// (sc->sigma_ready).  Block `first` reads that flag before each grid barrier
// and leaves its answer in sc->spec_go[t], which every block reads after the
// barrier, so all blocks stop after the same step.  sc->spec_done = the steps
// stored; returns that number, or -1 after a barrier timeout.
__device__ __forceinline__ int speculative_steps(const FilterArgs& a, int depth, int first, uint32_t members,
                                                 bool until_sigma, uint32_t& epoch, int* s_ok, float* s_cexp,
                                                 int* s_go) {
  const int n = a.n;
  const int gtid = (blockIdx.x - first) * blockDim.x + threadIdx.x;
  const int gstride = int(members) * blockDim.x;
  DevScalars* sc = a.sc;
  const float cexp = block_cexp(sc, s_cexp);
  int stored = depth;
  for (int t = 1; t <= depth; ++t) {
    const float4* src = t == 1 ? a.x0 : a.spec_x + size_t(t - 2) * size_t(a.cap);
    float4* dst = a.spec_x + size_t(t - 1) * size_t(a.cap);
    int32_t* z = a.spec_z + size_t(t - 1) * size_t(a.cap);
    // each point's own iterate and slots are loaded one trip ahead, so that
    // only the neighbour loads wait on the point before them
    StepHead next{};
    if (gtid < n) next = step_head<true>(a, src, gtid);
    for (int k = gtid; k < n; k += gstride) {
      const StepHead h = next;
      if (k + gstride < n) next = step_head<true>(a, src, k + gstride);
      const float4 xo =
          t == 1 ? eq5_step<true, true>(a, src, k, n, cexp, h) : eq5_step<false, true>(a, src, k, n, cexp, h);
      dst[k] = xo;
      z[k] = int32_t(sq3(xo));
    }
    const bool ask = until_sigma && t < depth;
    if (ask && blockIdx.x == first && threadIdx.x == 0) sc->spec_go[t] = ld_acquire_u32(&sc->sigma_ready) ? 0u : 1u;
    if (!grid_barrier(&sc->spec_barrier, &sc->status, members, epoch, s_ok, sc)) return -1;
    if (ask) {
      if (threadIdx.x == 0) *s_go = int(ld_acquire_u32(&sc->spec_go[t]));
      __syncthreads();
      const bool go = *s_go != 0;
      __syncthreads();
      if (!go) {
        stored = t;
        break;
      }
    }
  }
  if (gtid == 0) sc->spec_done = stored;
  return stored;
}

}  // namespace fgbd
