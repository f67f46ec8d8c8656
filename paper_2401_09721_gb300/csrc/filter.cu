// Graph low-pass filter (Eq. 5) and its FSLR selection (Eq. 6, Section 2.4) as
// a kernel of their own (k_filter, the device routine in select.cuh), the
// output of a chosen iterate in input order, and the graph / FSLR exports.
#include <algorithm>
#include <climits>

#include "select.cuh"

namespace fgbd {
namespace {

// NX further neighbour slots per point: 0 at window 1, 6 (w - 1) at window w
template <int NX>
__global__ void __launch_bounds__(kFilterThreads, 2) k_filter(FilterArgs a) {
  pdl_wait();
  // the stored steps count only if the noise-estimate launch finished them
  __shared__ int s_S;
  if (threadIdx.x == 0) {
    const int done = int(ld_acquire_u32(reinterpret_cast<const uint32_t*>(&a.sc->spec_done)));
    s_S = (a.mode == 0 && a.spec_depth > 0) ? min(done, a.spec_depth) : 0;
  }
  __syncthreads();
  uint32_t epoch = 0;
  select_filter<kFilterThreads, NX>(a, s_S, 0, gridDim.x, &a.sc->barrier, epoch);
}

// Segmented (window 1): frame f's blocks [start[f], start[f + 1]) select and
// filter frame f, with grid barriers among themselves only.
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS) k_filter_seg(const __grid_constant__ Seg<FilterArgs> s) {
  pdl_wait();
  const int f = seg_frame(s, blockIdx.x);
  const FilterArgs& a = s.a[f];
  __shared__ int s_S;
  if (threadIdx.x == 0) {
    const int done = int(ld_acquire_u32(reinterpret_cast<const uint32_t*>(&a.sc->spec_done)));
    s_S = (a.mode == 0 && a.spec_depth > 0) ? min(done, a.spec_depth) : 0;
  }
  __syncthreads();
  uint32_t epoch = 0;
  select_filter<THREADS, 0>(a, s_S, s.start[f], uint32_t(s.start[f + 1] - s.start[f]), &a.sc->barrier, epoch);
}

__global__ void __launch_bounds__(256) k_output(FilterArgs a) {
  pdl_wait();
  output_quads(a, a.sc->kept_buf, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------- export

constexpr int kMaxDegree = 6 * kMaxWindow;

__device__ __forceinline__ int gather_row(int k, int n, const GraphBufs& gb, int nb[kMaxDegree]) {
  int cnt = 0;
  if (!in_range(k, n)) return 0;
  const uint32_t pkk = gb.pk[k];
  const int4 s = gb.c4[k];
  const int slots = 6 + gb.nx;
  for (int j = 0; j < slots && j < kMaxDegree; ++j) {
    const int o = neighbour_of(j, k, n, pkk, s, gb.cx, gb.cx_stride);
    if (o >= 0) nb[cnt++] = o;
  }
  return cnt;
}

__global__ void k_csr_degree(int n, GraphBufs gb, int64_t* __restrict__ deg) {
  pdl_wait();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) {
    if (i == n) {
      deg[i] = 0;
      continue;
    }
    int nb[kMaxDegree];
    deg[i] = gather_row(gb.rank1[i], n, gb, nb);
  }
}

__global__ void k_csr_fill(int n, int bits, GraphBufs gb, const int64_t* __restrict__ row_ptr,
                           int32_t* __restrict__ col, float* __restrict__ w, int64_t col_capacity,
                           const DevScalars* __restrict__ sc) {
  pdl_wait();
  const double sg = sigma_g_of(sc);
  const float inv2 = sg > 0.0 ? float(1.0 / (sg * sg)) : 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int k = gb.rank1[i];
    int nb[kMaxDegree];
    const int cnt = gather_row(k, n, gb, nb);
    if (cnt == 0) continue;
    int orig[kMaxDegree];
    float wv[kMaxDegree];
    for (int j = 0; j < cnt; ++j) {
      orig[j] = gb.perm1[nb[j]];
      const float d2 = float(sq_dist_c1(gb.pk[k], gb.pk[nb[j]], bits));
      if (gb.node_sig && sc->sigma_mode == kSigmaPair) {
        // the pair reading: w_ij = exp(-d_ij^2 / (sigma_i sigma_j)); 1 where the product is 0
        const float s = gb.node_sig[k] * gb.node_sig[nb[j]];
        wv[j] = s > 0.f ? expf(-d2 / s) : 1.f;
      } else {
        wv[j] = expf(-d2 * inv2);
      }
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
  pdl_wait();
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
  pdl_wait();
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
  pdl_wait();
  const int64_t i = int64_t(blockIdx.x) * kScanBlock + threadIdx.x;
  if (i < count) data[i] += totals[blockIdx.x];
}

__global__ void k_spread_export(int n, const int32_t* __restrict__ rank1, const float* __restrict__ spread,
                                const uint8_t* __restrict__ keep8, float* __restrict__ spread_out,
                                uint8_t* __restrict__ keep_out) {
  pdl_wait();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int k = rank1[i];
    if (!in_range(k, n)) continue;
    if (spread_out) spread_out[i] = spread[k];
    if (keep_out) keep_out[i] = keep8[k] ? 1 : 0;
  }
}

}  // namespace

int filter_grid(int n, int num_sms, int nx) {
  int per_sm = 0;
  cudaError_t e;
  if (nx == extra_slots(3))
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter<extra_slots(3)>, kFilterThreads, 0);
  else if (nx == extra_slots(2))
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter<extra_slots(2)>, kFilterThreads, 0);
  else
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter<0>, kFilterThreads, 0);
  if (e != cudaSuccess || per_sm < 1) per_sm = 1;
  const int need = std::max(1, (n + kFilterThreads - 1) / kFilterThreads);
  return std::max(1, std::min(need, per_sm * num_sms));
}

cudaError_t launch_filter(const FilterArgs& a, int grid, cudaStream_t stream) {
  if (a.nx == extra_slots(2))
    return launch_kernel(k_filter<extra_slots(2)>, dim3(grid), dim3(kFilterThreads), 0, stream, true, a);
  if (a.nx == extra_slots(3))
    return launch_kernel(k_filter<extra_slots(3)>, dim3(grid), dim3(kFilterThreads), 0, stream, true, a);
  if (a.nx != 0) return cudaErrorInvalidValue;
  return launch_kernel(k_filter<0>, dim3(grid), dim3(kFilterThreads), 0, stream, true, a);
}

int filter_seg_max_per_sm(int threads) {
  int per_sm = 0;
  const cudaError_t e =
      threads == 256 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter_seg<256>, 256, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_filter_seg<512>, 512, 0);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return 1;
  }
  return per_sm;
}

cudaError_t launch_filter_seg(const FilterArgs* a, int count, int threads, int filter_per_sm, int num_sms,
                              cudaStream_t stream) {
  if (count < 1 || count > kSegMax || (threads != 256 && threads != 512)) return cudaErrorInvalidValue;
  for (int f = 0; f < count; ++f)
    if (a[f].nx != 0) return cudaErrorInvalidValue;
  // every block must be resident (grid barriers): at most the occupancy per SM
  const int per_sm = std::max(1, std::min(filter_per_sm, filter_seg_max_per_sm(threads)));
  const int pool = per_sm * num_sms;
  if (pool < count) return cudaErrorInvalidValue;
  Seg<FilterArgs> sg;
  int blocks[kSegMax];
  double total = 0.0;
  for (int f = 0; f < count; ++f) total += double(std::max(a[f].n, 1));
  int given = 0;
  for (int f = 0; f < count; ++f) {
    sg.a[f] = a[f];
    // in proportion to the points, at least one block, no more than one thread per point
    const int need = std::max(1, (a[f].n + threads - 1) / threads);
    const int left = count - 1 - f;
    int b = int(double(pool) * double(std::max(a[f].n, 1)) / total);
    b = std::max(1, std::min({b, need, pool - given - left}));
    given += b;
    blocks[f] = b;
  }
  const int grid = seg_layout(sg, blocks, count);
  if (threads == 256) return launch_kernel(k_filter_seg<256>, dim3(grid), dim3(256), 0, stream, true, sg);
  return launch_kernel(k_filter_seg<512>, dim3(grid), dim3(512), 0, stream, true, sg);
}

cudaError_t launch_output(const FilterArgs& a, cudaStream_t stream) {
  if (a.n <= 0) return cudaSuccess;
  const int grid = std::min((a.n + 255) / 256, 152 * 16);
  return launch_kernel(k_output, dim3(grid), dim3(256), 0, stream, false, a);
}

cudaError_t launch_csr_degree(int n, const GraphBufs& gb, int64_t* deg_out, cudaStream_t stream) {
  const int grid = std::max(1, std::min((n + 256) / 256, 152 * 16));
  return launch_kernel(k_csr_degree, dim3(grid), dim3(256), 0, stream, false, n, gb, deg_out);
}

cudaError_t launch_scan_i64(int64_t* data, int64_t count, int64_t* block_tmp, cudaStream_t stream) {
  if (count <= 0) return cudaSuccess;
  const int nb = int((count + kScanBlock - 1) / kScanBlock);
  {
    const cudaError_t le = launch_kernel(k_scan_blocks, dim3(nb), dim3(kScanBlock), 0, stream, false, data, count,
                                         block_tmp);
    if (le != cudaSuccess) return le;
  }
  {
    const cudaError_t le = launch_kernel(k_scan_totals, dim3(1), dim3(32), 0, stream, false, block_tmp, nb);
    if (le != cudaSuccess) return le;
  }
  return launch_kernel(k_scan_add, dim3(nb), dim3(kScanBlock), 0, stream, false, data, count, block_tmp);
}

cudaError_t launch_csr_fill(int n, int bits, const GraphBufs& gb, const int64_t* row_ptr, int32_t* col,
                            float* w, int64_t col_capacity, const DevScalars* sc, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = std::min((n + 255) / 256, 152 * 16);
  return launch_kernel(k_csr_fill, dim3(grid), dim3(256), 0, stream, false, n, bits, gb, row_ptr, col, w,
                       col_capacity, sc);
}

cudaError_t launch_spread_export(int n, const int32_t* rank1, const float* spread, const uint8_t* keep8,
                                 float* spread_out, uint8_t* keep_out, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = std::min((n + 255) / 256, 152 * 16);
  return launch_kernel(k_spread_export, dim3(grid), dim3(256), 0, stream, false, n, rank1, spread, keep8, spread_out,
                       keep_out);
}

}  // namespace fgbd
