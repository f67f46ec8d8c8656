// Differentiable graph filter: Eq. 5 generalised to a filter strength alpha
// and a weight bandwidth sigma, with its adjoint.
//
//   x_{t+1} = (1 - alpha) x_t + alpha R x_t,   R = D^{-1} W,
//   W_ij = exp(-d_ij^2 / sigma^2) over the scan-line graph (Eq. 4),
// so alpha = 1/2 and sigma = sigma_g give Eq. 5 (W_g = D + W, D_g = 2D).  For a
// loss L(x_q) with g = dL/dx_q and u_t = dL/dx_t:
//   u_t = P^T u_{t+1} = (1 - alpha) u_{t+1} + alpha W D^{-1} u_{t+1}
//   dL/dalpha = sum_t u_{t+1} . (R x_t - x_t)
//   dL/dsigma = sum_t alpha u_{t+1} . (dR/dsigma) x_t,
//   (dR/dsigma x)_i = (2 / sigma^3) sum_j R_ij (d_ij^2 - e_i) x_j,
//   e_i = sum_j R_ij d_ij^2
// (the derivative of a row-normalised Gaussian row; the row-minimum shift
// used against underflow cancels in it).  The rows of R and, for the
// adjoint, the weight of i in each neighbour's row (R^T) are tabulated once
// per forward call.  Iterates are kept every `checkpoint` steps and the ones
// in between are recomputed segment by segment in the backward call.
// Reductions are float64 per block, summed in a fixed order: deterministic.
#include <algorithm>
#include <climits>

#include "fgbd_internal.cuh"

namespace fgbd {
namespace {

constexpr int kDiffThreads = 256;

__device__ __forceinline__ double diff_sigma(double sigma, const DevScalars* sc) {
  return sigma > 0.0 ? sigma : sigma_g_of(sc);
}

// Rows of R: neighbours (C1 k-1, k+1, then the C2/C3 slots; -1 unused),
// normalised weights, squared distances and their R-weighted mean e_i.
__global__ void __launch_bounds__(kDiffThreads)
    k_diff_rows(int n, int bits, double sigma_in, const uint32_t* __restrict__ pk, const int4* __restrict__ c4,
                const DevScalars* __restrict__ sc, int32_t* __restrict__ nb, float* __restrict__ R,
                float* __restrict__ d2f, float* __restrict__ e) {
  pdl_wait();
  // the exponent scale once per block (float64 is slow on this GPU)
  __shared__ float s_cexp;
  if (threadIdx.x == 0) {
    const double sg = diff_sigma(sigma_in, sc);
    s_cexp = sg > 0.0 ? float(1.4426950408889634 / (sg * sg)) : 0.f;
  }
  __syncthreads();
  const float cexp = s_cexp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int j[kK];
    const uint32_t ci = pk[i];  // packed code, with the same-line variant's missing-C1-link bits
    j[0] = c1_prev_linked(ci, i) ? i - 1 : -1;
    j[1] = c1_next_linked(ci, i, n) ? i + 1 : -1;
    const int4 s = c4[i];
    j[2] = in_range(s.x, n) ? s.x : -1;
    j[3] = in_range(s.y, n) ? s.y : -1;
    j[4] = in_range(s.z, n) ? s.z : -1;
    j[5] = in_range(s.w, n) ? s.w : -1;
    int d2[kK];
    int dmin = INT_MAX;
#pragma unroll
    for (int t = 0; t < kK; ++t) {
      d2[t] = j[t] >= 0 ? sq_dist_c1(ci, pk[j[t]], bits) : INT_MAX;
      dmin = min(dmin, d2[t]);
    }
    float w[kK];
    float sw = 0.f;
#pragma unroll
    for (int t = 0; t < kK; ++t) {
      w[t] = j[t] >= 0 ? exp2f(float(dmin - d2[t]) * cexp) : 0.f;
      sw += w[t];
    }
    if (sw == 0.f) {
      // no neighbour (a one-point graph): R x = x, as Eq. 5 leaves such a point unchanged
      j[0] = i;
      d2[0] = 0;
      w[0] = 1.f;
      sw = 1.f;
    }
    const float inv = 1.f / sw;
    float ei = 0.f;
#pragma unroll
    for (int t = 0; t < kK; ++t) {
      const float r = w[t] * inv;
      nb[size_t(i) * kK + t] = j[t];
      R[size_t(i) * kK + t] = r;
      d2f[size_t(i) * kK + t] = j[t] >= 0 ? float(d2[t]) : 0.f;
      ei = fmaf(r, j[t] >= 0 ? float(d2[t]) : 0.f, ei);
    }
    e[i] = ei;
  }
}

// RT[i][t] = R[j][s] for j = nb[i][t] and nb[j][s] = i: the weight of i in
// its neighbour's row (the graph is symmetric, so the slot exists).
__global__ void __launch_bounds__(kDiffThreads)
    k_diff_rows_t(int n, const int32_t* __restrict__ nb, const float* __restrict__ R, float* __restrict__ RT) {
  pdl_wait();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
    for (int t = 0; t < kK; ++t) {
      const int j = nb[size_t(i) * kK + t];
      float v = 0.f;
      if (in_range(j, n)) {
#pragma unroll
        for (int s = 0; s < kK; ++s)
          if (nb[size_t(j) * kK + s] == i) v = R[size_t(j) * kK + s];
      }
      RT[size_t(i) * kK + t] = v;
    }
  }
}

// x[k] = rgb[perm1[k]] (input order -> sorted order)
__global__ void __launch_bounds__(kDiffThreads)
    k_diff_gather(int n, const float* __restrict__ rgb, const int32_t* __restrict__ perm1, float4* __restrict__ x) {
  pdl_wait();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int i = perm1[k];
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (in_range(i, n)) v = make_float4(rgb[3 * size_t(i)], rgb[3 * size_t(i) + 1], rgb[3 * size_t(i) + 2], 0.f);
    x[k] = v;
  }
}

// out[perm1[k]] = x[k] (sorted order -> input order)
__global__ void __launch_bounds__(kDiffThreads)
    k_diff_scatter(int n, const float4* __restrict__ x, const int32_t* __restrict__ perm1, float* __restrict__ out) {
  pdl_wait();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int i = perm1[k];
    if (!in_range(i, n)) continue;
    const float4 v = x[k];
    out[3 * size_t(i)] = v.x;
    out[3 * size_t(i) + 1] = v.y;
    out[3 * size_t(i) + 2] = v.z;
  }
}

// One forward step: dst = (1 - alpha) src + alpha R src
__global__ void __launch_bounds__(kDiffThreads)
    k_diff_step(int n, float alpha, const int32_t* __restrict__ nb, const float* __restrict__ R,
                const float4* __restrict__ src, float4* __restrict__ dst) {
  pdl_wait();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float rx = 0.f, ry = 0.f, rz = 0.f;
#pragma unroll
    for (int t = 0; t < kK; ++t) {
      const int j = nb[size_t(i) * kK + t];
      if (in_range(j, n)) {
        const float r = R[size_t(i) * kK + t];
        const float4 v = src[j];
        rx = fmaf(r, v.x, rx);
        ry = fmaf(r, v.y, ry);
        rz = fmaf(r, v.z, rz);
      }
    }
    const float4 s = src[i];
    const float a = 1.f - alpha;
    dst[i] = make_float4(fmaf(a, s.x, alpha * rx), fmaf(a, s.y, alpha * ry), fmaf(a, s.z, alpha * rz), 0.f);
  }
}

// Float-float accumulator (hi + lo): TwoSum (Knuth) and the TwoProduct of a
// fused multiply-add keep products and sums of float32 values exact to about
// 44 bits without float64, which is slow on this GPU.
struct FF2 {
  float hi, lo;
};
__device__ __forceinline__ FF2 ff2_add(FF2 x, FF2 y) {
  const float s = __fadd_rn(x.hi, y.hi);
  const float bb = __fsub_rn(s, x.hi);
  const float err = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));
  const float lo = __fadd_rn(err, __fadd_rn(x.lo, y.lo));
  const float h = __fadd_rn(s, lo);
  return {h, __fsub_rn(lo, __fsub_rn(h, s))};
}
// x += a * b, the product exact
__device__ __forceinline__ FF2 ff2_fma(FF2 x, float a, float b) {
  const float p = __fmul_rn(a, b);
  return ff2_add(x, {p, fmaf(a, b, -p)});
}
__device__ __forceinline__ FF2 ff2_shfl_down(FF2 x, int o) {
  return {__shfl_down_sync(0xffffffffu, x.hi, o), __shfl_down_sync(0xffffffffu, x.lo, o)};
}

// One adjoint step: u_out = P^T u, and this step's terms of dL/dalpha and
// dL/dsigma (per block, float64) at partial[2 * blockIdx.x + {0, 1}].  The
// per-point terms are accumulated in float-float and only the block's warp
// sums are combined in float64.
__global__ void __launch_bounds__(kDiffThreads)
    k_diff_back_step(int n, float alpha, double sigma_in, const int32_t* __restrict__ nb,
                     const float* __restrict__ R, const float* __restrict__ RT, const float* __restrict__ d2f,
                     const float* __restrict__ e, const float4* __restrict__ x, const float4* __restrict__ u,
                     float4* __restrict__ u_out, const DevScalars* __restrict__ sc, double* __restrict__ partial) {
  pdl_wait();
  __shared__ FF2 s_red[2][kDiffThreads / 32];
  __shared__ double s_scale;  // alpha * 2 / sigma^3
  if (threadIdx.x == 0) {
    const double sg = diff_sigma(sigma_in, sc);
    s_scale = sg > 0.0 ? double(alpha) * (2.0 / (sg * sg * sg)) : 0.0;
  }
  FF2 da = {0.f, 0.f}, ds = {0.f, 0.f};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float ux = 0.f, uy = 0.f, uz = 0.f;  // (W D^-1 u)_i
    float rx = 0.f, ry = 0.f, rz = 0.f;  // (R x)_i
    float gx = 0.f, gy = 0.f, gz = 0.f;  // sum_j R_ij (d2_ij - e_i) x_j
    const float ei = e[i];
#pragma unroll
    for (int t = 0; t < kK; ++t) {
      const int j = nb[size_t(i) * kK + t];
      if (in_range(j, n)) {
        const float rt = RT[size_t(i) * kK + t];
        const float r = R[size_t(i) * kK + t];
        const float dd = r * (d2f[size_t(i) * kK + t] - ei);
        const float4 uj = u[j];
        const float4 xj = x[j];
        ux = fmaf(rt, uj.x, ux);
        uy = fmaf(rt, uj.y, uy);
        uz = fmaf(rt, uj.z, uz);
        rx = fmaf(r, xj.x, rx);
        ry = fmaf(r, xj.y, ry);
        rz = fmaf(r, xj.z, rz);
        gx = fmaf(dd, xj.x, gx);
        gy = fmaf(dd, xj.y, gy);
        gz = fmaf(dd, xj.z, gz);
      }
    }
    const float4 ui = u[i];
    const float4 xi = x[i];
    const float a = 1.f - alpha;
    u_out[i] = make_float4(fmaf(a, ui.x, alpha * ux), fmaf(a, ui.y, alpha * uy), fmaf(a, ui.z, alpha * uz), 0.f);
    da = ff2_fma(ff2_fma(ff2_fma(da, ui.x, rx - xi.x), ui.y, ry - xi.y), ui.z, rz - xi.z);
    ds = ff2_fma(ff2_fma(ff2_fma(ds, ui.x, gx), ui.y, gy), ui.z, gz);
  }
  // block sums in a fixed order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    da = ff2_add(da, ff2_shfl_down(da, o));
    ds = ff2_add(ds, ff2_shfl_down(ds, o));
  }
  if (lane == 0) {
    s_red[0][warp] = da;
    s_red[1][warp] = ds;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a0 = 0.0, a1 = 0.0;
    for (int w = 0; w < kDiffThreads / 32; ++w) {
      a0 += double(s_red[0][w].hi) + double(s_red[0][w].lo);
      a1 += double(s_red[1][w].hi) + double(s_red[1][w].lo);
    }
    partial[2 * blockIdx.x] = a0;
    partial[2 * blockIdx.x + 1] = a1 * s_scale;
  }
}

// grad[0..1] = the sums of `count` (dalpha, dsigma) partials, in a fixed order
__global__ void __launch_bounds__(256) k_diff_reduce(int count, const double* __restrict__ partial,
                                                     double* __restrict__ grad) {
  pdl_wait();
  __shared__ double s[2][256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    a += partial[2 * i];
    b += partial[2 * i + 1];
  }
  s[0][threadIdx.x] = a;
  s[1][threadIdx.x] = b;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s[0][threadIdx.x] += s[0][threadIdx.x + o];
      s[1][threadIdx.x] += s[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    grad[0] = s[0][0];
    grad[1] = s[1][0];
  }
}

}  // namespace

int diff_grid(int n, int num_sms) { return std::max(1, std::min((n + kDiffThreads - 1) / kDiffThreads, num_sms * 8)); }

cudaError_t launch_diff_rows(int n, int bits, double sigma, const GraphBufs& gb, const DevScalars* sc,
                             const DiffBufs& db, int num_sms, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = diff_grid(n, num_sms);
  {
    const cudaError_t le = launch_kernel(k_diff_rows, dim3(grid), dim3(kDiffThreads), 0, stream, false, n, bits,
                                         sigma, gb.pk, gb.c4, sc, db.nb, db.R, db.d2, db.e);
    if (le != cudaSuccess) return le;
  }
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  return launch_kernel(k_diff_rows_t, dim3(grid), dim3(kDiffThreads), 0, stream, false, n, db.nb, db.R, db.RT);
}

cudaError_t launch_diff_gather(int n, const float* rgb, const int32_t* perm1, float4* x, int num_sms,
                               cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  return launch_kernel(k_diff_gather, dim3(diff_grid(n, num_sms)), dim3(kDiffThreads), 0, stream, false, n, rgb,
                       perm1, x);
}

cudaError_t launch_diff_scatter(int n, const float4* x, const int32_t* perm1, float* out, int num_sms,
                                cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  return launch_kernel(k_diff_scatter, dim3(diff_grid(n, num_sms)), dim3(kDiffThreads), 0, stream, false, n, x, perm1,
                       out);
}

cudaError_t launch_diff_step(int n, float alpha, const DiffBufs& db, const float4* src, float4* dst, int num_sms,
                             cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  return launch_kernel(k_diff_step, dim3(diff_grid(n, num_sms)), dim3(kDiffThreads), 0, stream, false, n, alpha,
                       db.nb, db.R, src, dst);
}

cudaError_t launch_diff_back_step(int n, float alpha, double sigma, const DiffBufs& db, const float4* x,
                                  const float4* u, float4* u_out, const DevScalars* sc, double* partial,
                                  int num_sms, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  return launch_kernel(k_diff_back_step, dim3(diff_grid(n, num_sms)), dim3(kDiffThreads), 0, stream, false, n, alpha,
                       sigma, db.nb, db.R, db.RT, db.d2, db.e, x, u, u_out, sc, partial);
}

cudaError_t launch_diff_reduce(int count, const double* partial, double* grad, cudaStream_t stream) {
  return launch_kernel(k_diff_reduce, dim3(1), dim3(256), 0, stream, false, count, partial, grad);
}

}  // namespace fgbd
