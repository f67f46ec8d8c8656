// Graph low-pass filter (Eq. 5) and its FSLR selection (Eq. 6, Section 2.4).
//
// k_filter is one cooperative launch over all points, in sorted order:
//   phase 0   the FSLR keep flag of each point (spread <= 2 sigma_est) goes to
//             keep8; the kept power sum y^2 and the kept count are reduced;
//             x_0 = y is written unless the first steps are stored already.
//   step t    x_t = x_{t-1}/2 + (sum_j e_j x_{t-1}[j]) / (2 sum_j e_j) with
//             e_j = exp(-(d2_j - min_j d2_j) / sigma_g^2) (eq5_step): the rows
//             of D^{-1} W of Eq. 4, computed on the fly from the neighbours'
//             coordinates (carried in x.w), so no weight array is read.
//             In select mode the kept power sum x_t^2 is reduced and, after a
//             grid barrier, every block evaluates the same
//             J(t) = |sigma^2 - (sum y^2 - sum x_t^2)/(3 N_sel)| and stops at
//             the first t with J(t) >= J(t-1), keeping q* = t-1.
//   output    the kept iterate is gathered back to input order (optional).
// The steps do not depend on sigma_est, only the keep flags and J do: the
// noise-estimate launch stores x_1..x_S and each point's Eq. 6 term
// y^2 - x_q^2 (speculative_steps), and phase 0 then also reduces those terms
// over the kept points, so J(1..S) need no step here; ordinary steps continue
// from x_S only if J still falls there.
// Sums of squares are fixed-point integers (2^-8), so the reduction is exact
// and independent of the order in which blocks add.
// The grid barrier is a counter with a 2 s wait limit; a block that gives up
// latches kFlagTimeout and every block returns.
#include <algorithm>
#include <climits>

#include "filter_step.cuh"

namespace fgbd {
namespace {

// float64 spread of point k, used only where the float32 value is too close to
// the threshold to decide (Section 2.4: mean of the three population stds)
__device__ double spread_f64(const FilterArgs& a, int k) {
  int nb[7];
  int cnt = 0;
  nb[cnt++] = k;
  if (k > 0) nb[cnt++] = k - 1;
  if (k + 1 < a.n) nb[cnt++] = k + 1;
  const int4 s = a.c4[k];
  if (in_range(s.x, a.n)) nb[cnt++] = s.x;
  if (in_range(s.y, a.n)) nb[cnt++] = s.y;
  if (in_range(s.z, a.n)) nb[cnt++] = s.z;
  if (in_range(s.w, a.n)) nb[cnt++] = s.w;
  double mean[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < cnt; ++j) {
    float r, g, b;
    load_y(a, nb[j], r, g, b);
    mean[0] += r;
    mean[1] += g;
    mean[2] += b;
  }
  for (int c = 0; c < 3; ++c) mean[c] /= double(cnt);
  double var[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < cnt; ++j) {
    float r, g, b;
    load_y(a, nb[j], r, g, b);
    var[0] += (r - mean[0]) * (r - mean[0]);
    var[1] += (g - mean[1]) * (g - mean[1]);
    var[2] += (b - mean[2]) * (b - mean[2]);
  }
  return (sqrt(var[0] / cnt) + sqrt(var[1] / cnt) + sqrt(var[2] / cnt)) / 3.0;
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
  if (kept >= 2) return __ldcg(&a.spec_x[size_t(kept - 2) * size_t(a.cap) + k]);
  return __ldcg(&(kept ? a.xbuf1 : a.xbuf0)[k]);
}

// Sums of several 64-bit values over the block (two's complement: exact in any order)
template <int K>
__device__ __forceinline__ void block_sums(unsigned long long (&v)[K], unsigned long long* s_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < K; ++i) v[i] = warp_sum(v[i]);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < K; ++i) s_red[i * (kFilterThreads / 32) + warp] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < K) {
    unsigned long long t = 0;
    for (int w = 0; w < kFilterThreads / 32; ++w) t += s_red[threadIdx.x * (kFilterThreads / 32) + w];
    s_red[K * (kFilterThreads / 32) + threadIdx.x] = t;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < K; ++i) v[i] = s_red[K * (kFilterThreads / 32) + i];
  __syncthreads();
}

constexpr int kSums = 3 + 2 * kSpecMax;  // kept y^2, all y^2, kept count, then per stored step kept and all terms

__global__ void __launch_bounds__(kFilterThreads, 2) k_filter(FilterArgs a) {
  __shared__ unsigned long long s_red[(kSums + 1) * (kFilterThreads / 32)];
  __shared__ int s_ok;
  __shared__ double s_J;
  uint32_t epoch = 0;
  const int n = a.n;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int gstride = gridDim.x * blockDim.x;
  DevScalars* sc = a.sc;
  const bool select = a.mode == 0;
  // the stored steps count only if the noise-estimate launch finished them
  const int S = (select && a.spec_depth > 0 &&
                 ld_acquire_u32(reinterpret_cast<const uint32_t*>(&sc->spec_done)) == uint32_t(a.spec_depth))
                    ? a.spec_depth
                    : 0;

  double sigma = 0.0;
  float t_lo = 0.f, t_hi = 0.f;
  double thr = 0.0;
  if (select) {
    sigma = *a.sigma_src;
    thr = a.fslr_factor * sigma;
    const double band = a.dtype == 0 ? 2e-6 : 5e-5;
    t_lo = float(thr * (1.0 - band));
    t_hi = float(thr * (1.0 + band));
  }

  // ---- phase 0: keep flags and the Eq. 6 sums; x_0 = y unless the steps are stored
  unsigned long long acc[kSums] = {};
  for (int k = gtid; k < n; k += gstride) {
    const float4 x0 = x0_of(a, k);
    if (!S) a.xbuf0[k] = x0;
    if (select) {
      const float sp = a.spread[k];
      bool keep;
      if (a.all_points || sp <= t_lo) keep = true;
      else if (sp > t_hi) keep = false;
      else keep = !(spread_f64(a, k) > thr);
      a.keep8[k] = keep ? 1 : 0;
      const unsigned long long q2 = sq3(x0);
      acc[1] += q2;
      if (keep) {
        acc[0] += q2;
        acc[2] += 1;
      }
    }
  }
  // the stored steps' Eq. 6 terms (a second pass: this thread's own keep flags)
  if (S > 0) {
    for (int k = gtid; k < n; k += gstride) {
      const bool keep = a.keep8[k] != 0;
#pragma unroll
      for (int q = 0; q < kSpecMax; ++q) {
        if (q < S) {
          const unsigned long long z = (unsigned long long)(long long)a.spec_z[size_t(q) * size_t(a.cap) + k];
          acc[4 + 2 * q] += z;
          if (keep) acc[3 + 2 * q] += z;
        }
      }
    }
  }
  if (select) {
    block_sums<kSums>(acc, s_red);
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
  if (!grid_barrier(&sc->barrier, &sc->status, gridDim.x, epoch, &s_ok)) return;

  bool keep_all = false;
  unsigned long long ysq = 0;
  double nsel = 1.0;
  if (select) {
    const unsigned long long nkt = ld_relaxed_u64(&sc->n_keep);
    keep_all = nkt == 0;  // no point left: every point is used
    nsel = keep_all ? double(n) : double(nkt);
    ysq = keep_all ? ld_relaxed_u64(&sc->ysq_all) : ld_relaxed_u64(&sc->ysq_keep);
  }
  const float cexp = step_cexp(sc);

  double J_prev = sigma * sigma;  // J(0): nothing filtered yet
  if (select && gtid == 0) sc->J[0] = J_prev;
  int q_final = 0;
  bool stopped = false;
  const int q_fixed = a.q_src ? min(max(*a.q_src, 0), kQCap) : a.q_fixed;
  const int q_limit = n == 0 ? 0 : (select ? a.q_max : q_fixed);
  // J(1..S) from the stored terms
  for (int t = 1; t <= min(S, q_limit); ++t) {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(keep_all ? &sc->spec_all[t]
                                                                                          : &sc->spec_keep[t]);
    const double lost = double((long long)ld_relaxed_u64(src)) * (1.0 / double(1 << kSqShift));
    const double J = fabs(sigma * sigma - lost / (3.0 * nsel));
    if (gtid == 0) {
      sc->J[t] = J;
      sc->n_J = t + 1;
    }
    if (J >= J_prev) {
      q_final = t - 1;
      stopped = true;
      break;
    }
    J_prev = J;
    q_final = t;
  }
  for (int t = S + 1; t <= q_limit && !stopped; ++t) {
    const float4* __restrict__ src =
        (S > 0 && t == S + 1) ? a.spec_x + size_t(S - 1) * size_t(a.cap) : ((t & 1) ? a.xbuf0 : a.xbuf1);
    float4* __restrict__ dst = (t & 1) ? a.xbuf1 : a.xbuf0;
    unsigned long long loc = 0;
    for (int k = gtid; k < n; k += gstride) {
      const float4 xo = eq5_step(a, src, k, n, cexp);
      dst[k] = xo;
      if (select && (keep_all || a.keep8[k])) loc += sq3(xo);
    }
    if (select) {
      loc = block_sum_u64<kFilterThreads>(loc, s_red);
      if (threadIdx.x == 0 && loc) atomicAdd(&sc->sumsq[t], loc);
    }
    if (!grid_barrier(&sc->barrier, &sc->status, gridDim.x, epoch, &s_ok)) return;
    if (select) {
      if (threadIdx.x == 0) {
        const unsigned long long ss = ld_relaxed_u64(&sc->sumsq[t]);
        const double lost = double((long long)(ysq - ss)) * (1.0 / double(1 << kSqShift));
        s_J = fabs(sigma * sigma - lost / (3.0 * nsel));
      }
      __syncthreads();
      const double J = s_J;
      if (gtid == 0) sc->J[t] = J;
      if (J >= J_prev) {
        q_final = t - 1;
        if (gtid == 0) sc->n_J = t + 1;
        break;
      }
      J_prev = J;
      q_final = t;
      if (gtid == 0) sc->n_J = t + 1;
    } else {
      q_final = t;
    }
  }
  // where the kept iterate is
  const int kept = (S > 0 && q_final <= S) ? (q_final == 0 ? -1 : 2 + q_final - 1) : (q_final & 1);
  if (gtid == 0) {
    if (!a.q_src) sc->q_sel = q_final;
    sc->kept_buf = kept;
    if (select) sc->sel_valid = 1;
    if (select && q_limit == 0) sc->n_J = 1;
  }
  if (a.out) {
    for (int i = gtid; i < n; i += gstride) {
      const int k = a.rank1[i];
      if (!in_range(k, n)) continue;
      write_out(a, i, kept_value(a, kept, k));
    }
  }
}

__global__ void __launch_bounds__(256) k_output(FilterArgs a) {
  const int kept = a.sc->kept_buf;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += gridDim.x * blockDim.x) {
    const int k = a.rank1[i];
    if (!in_range(k, a.n)) continue;
    write_out(a, i, kept_value(a, kept, k));
  }
}

// ---------------------------------------------------------------- export

__device__ __forceinline__ int gather_row(int k, int n, const int4* c4, int nb[6]) {
  int cnt = 0;
  if (!in_range(k, n)) return 0;
  if (k > 0) nb[cnt++] = k - 1;
  if (k + 1 < n) nb[cnt++] = k + 1;
  const int4 s = c4[k];
  if (in_range(s.x, n)) nb[cnt++] = s.x;
  if (in_range(s.y, n)) nb[cnt++] = s.y;
  if (in_range(s.z, n)) nb[cnt++] = s.z;
  if (in_range(s.w, n)) nb[cnt++] = s.w;
  return cnt;
}

__global__ void k_csr_degree(int n, const int32_t* __restrict__ rank1, const int4* __restrict__ c4,
                             int64_t* __restrict__ deg) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) {
    if (i == n) {
      deg[i] = 0;
      continue;
    }
    int nb[6];
    deg[i] = gather_row(rank1[i], n, c4, nb);
  }
}

__global__ void k_csr_fill(int n, int bits, const int32_t* __restrict__ rank1,
                           const int32_t* __restrict__ perm1, const uint32_t* __restrict__ pk,
                           const int4* __restrict__ c4, const int64_t* __restrict__ row_ptr,
                           int32_t* __restrict__ col, float* __restrict__ w, int64_t col_capacity,
                           const DevScalars* __restrict__ sc) {
  const double sg = sigma_g_of(sc);
  const float inv2 = sg > 0.0 ? float(1.0 / (sg * sg)) : 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int k = rank1[i];
    int nb[6];
    const int cnt = gather_row(k, n, c4, nb);
    if (cnt == 0) continue;
    int orig[6];
    float wv[6];
    for (int j = 0; j < cnt; ++j) {
      orig[j] = perm1[nb[j]];
      wv[j] = expf(-float(sq_dist_c1(pk[k], pk[nb[j]], bits)) * inv2);
    }
    for (int a = 1; a < cnt; ++a) {  // insertion sort by input index
      const int o = orig[a];
      const float x = wv[a];
      int b = a - 1;
      while (b >= 0 && orig[b] > o) {
        orig[b + 1] = orig[b];
        wv[b + 1] = wv[b];
        --b;
      }
      orig[b + 1] = o;
      wv[b + 1] = x;
    }
    const int64_t base = row_ptr[i];
    if (base < 0 || base + cnt > col_capacity) continue;
    for (int j = 0; j < cnt; ++j) {
      col[base + j] = orig[j];
      if (w) w[base + j] = wv[j];
    }
  }
}

// exclusive scan of int64 in place: per-block scans, scan of block totals, add
constexpr int kScanBlock = 1024;

__global__ void k_scan_blocks(int64_t* data, int64_t count, int64_t* totals) {
  __shared__ int64_t s[kScanBlock];
  const int64_t i = int64_t(blockIdx.x) * kScanBlock + threadIdx.x;
  const int64_t v = i < count ? data[i] : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < kScanBlock; o <<= 1) {
    const int64_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < count) data[i] = s[threadIdx.x] - v;
  if (threadIdx.x == kScanBlock - 1) totals[blockIdx.x] = s[threadIdx.x];
}

__global__ void k_scan_totals(int64_t* totals, int nb) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int64_t run = 0;
    for (int b = 0; b < nb; ++b) {
      const int64_t t = totals[b];
      totals[b] = run;
      run += t;
    }
  }
}

__global__ void k_scan_add(int64_t* data, int64_t count, const int64_t* totals) {
  const int64_t i = int64_t(blockIdx.x) * kScanBlock + threadIdx.x;
  if (i < count) data[i] += totals[blockIdx.x];
}

__global__ void k_spread_export(int n, const int32_t* __restrict__ rank1, const float* __restrict__ spread,
                                const uint8_t* __restrict__ keep8, float* __restrict__ spread_out,
                                uint8_t* __restrict__ keep_out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int k = rank1[i];
    if (!in_range(k, n)) continue;
    if (spread_out) spread_out[i] = spread[k];
    if (keep_out) keep_out[i] = keep8[k] ? 1 : 0;
  }
}

}  // namespace

int filter_grid(int n, int num_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter, kFilterThreads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int need = std::max(1, (n + kFilterThreads - 1) / kFilterThreads);
  return std::max(1, std::min(need, per_sm * num_sms));
}

cudaError_t launch_filter(const FilterArgs& a, int grid, cudaStream_t stream) {
  FilterArgs copy = a;
  void* args[] = {&copy};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_filter), dim3(grid),
                                     dim3(kFilterThreads), args, 0, stream);
}

cudaError_t launch_output(const FilterArgs& a, cudaStream_t stream) {
  if (a.n <= 0) return cudaSuccess;
  const int grid = std::min((a.n + 255) / 256, 152 * 16);
  k_output<<<grid, 256, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_csr_degree(int n, const GraphBufs& gb, int64_t* deg_out, cudaStream_t stream) {
  const int grid = std::max(1, std::min((n + 256) / 256, 152 * 16));
  k_csr_degree<<<grid, 256, 0, stream>>>(n, gb.rank1, gb.c4, deg_out);
  return cudaGetLastError();
}

cudaError_t launch_scan_i64(int64_t* data, int64_t count, int64_t* block_tmp, cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  const int nb = int((count + kScanBlock - 1) / kScanBlock);
  k_scan_blocks<<<nb, kScanBlock, 0, stream>>>(data, count, block_tmp);
  k_scan_totals<<<1, 32, 0, stream>>>(block_tmp, nb);
  k_scan_add<<<nb, kScanBlock, 0, stream>>>(data, count, block_tmp);
  return cudaGetLastError();
}

cudaError_t launch_csr_fill(int n, int bits, const GraphBufs& gb, const int64_t* row_ptr, int32_t* col,
                            float* w, int64_t col_capacity, const DevScalars* sc, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = std::min((n + 255) / 256, 152 * 16);
  k_csr_fill<<<grid, 256, 0, stream>>>(n, bits, gb.rank1, gb.perm1, gb.pk, gb.c4, row_ptr, col, w, col_capacity, sc);
  return cudaGetLastError();
}

cudaError_t launch_spread_export(int n, const int32_t* rank1, const float* spread, const uint8_t* keep8,
                                 float* spread_out, uint8_t* keep_out, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = std::min((n + 255) / 256, 152 * 16);
  k_spread_export<<<grid, 256, 0, stream>>>(n, rank1, spread, keep8, spread_out, keep_out);
  return cudaGetLastError();
}

}  // namespace fgbd
