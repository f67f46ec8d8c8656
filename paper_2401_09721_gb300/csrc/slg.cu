// SLG: scan-line graph construction (Section 2.2).
//
// 1. k_hist: scan-line codes C1..C3 (Eq. 1-3) of every point and the digit
//    histograms of every radix pass of every code, in one read of xyz.
// 2. k_sort_pass: one least-significant-digit pass of a stable onesweep radix
//    sort over all three codes at once (8-bit digits, dynamic tile ids,
//    decoupled look-back with a time-bounded wait).  Ties keep input order,
//    so equal codes are ordered by index.  The last pass writes the orders,
//    the packed C1 code of each sorted point, and the C1/C2 rank of each
//    input point.
// 3. k_link: points consecutive along a code are linked (Section 2.2).  In C1
//    order the code-1 neighbours are implicit (k-1, k+1); C2/C3 neighbours
//    are written as slots, a pair already linked by an earlier code is left
//    out so the union is a set, and each distinct edge's length is summed
//    for sigma_g.
#include <algorithm>

#include "fgbd_internal.cuh"

namespace fgbd {
namespace {

constexpr uint32_t kLbAgg = 1u << 30;
constexpr uint32_t kLbPre = 2u << 30;
constexpr uint32_t kLbFlags = 3u << 30;
constexpr uint32_t kLbCount = kLbAgg - 1u;

__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_gpu(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// exclusive scan of one value per thread over a 256-thread block
__device__ __forceinline__ uint32_t block_exclusive_scan_256(uint32_t v, uint32_t* s_warp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  uint32_t off = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) off += (w < warp) ? s_warp[w] : 0u;
  __syncthreads();
  return off + x - v;
}

__global__ void __launch_bounds__(256) k_hist(const int32_t* __restrict__ xyz, int n, int bits,
                                              int passes, uint32_t* __restrict__ zero_buf,
                                              size_t zero_words, DevScalars* __restrict__ sc) {
  __shared__ uint32_t h[3][kMaxPasses][kRadix];
  uint32_t* hf = &h[0][0][0];
  for (int i = threadIdx.x; i < 3 * kMaxPasses * kRadix; i += blockDim.x) hf[i] = 0;
  const size_t gtid = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const size_t gstride = size_t(gridDim.x) * blockDim.x;
  for (size_t i = gtid; i < zero_words; i += gstride) zero_buf[i] = 0;
  __syncthreads();
  const uint32_t m = (1u << bits) - 1u;
  bool bad = false;
  for (size_t i = gtid; i < size_t(n); i += gstride) {
    const int xi = xyz[3 * i], yi = xyz[3 * i + 1], zi = xyz[3 * i + 2];
    bad |= (uint32_t(xi) > m) | (uint32_t(yi) > m) | (uint32_t(zi) > m);
    const uint32_t x = uint32_t(xi) & m, y = uint32_t(yi) & m, z = uint32_t(zi) & m;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const uint32_t key = code_of(c, x, y, z, bits);
      for (int p = 0; p < passes; ++p) atomicAdd(&h[c][p][(key >> (kRadixBits * p)) & (kRadix - 1)], 1u);
    }
  }
  if (bad) atomicOr(&sc->status, kFlagRange);
  __syncthreads();
  for (int i = threadIdx.x; i < 3 * kMaxPasses * kRadix; i += blockDim.x) {
    const uint32_t v = hf[i];
    if (v) atomicAdd(&sc->hist[0][0][0] + i, v);
  }
}

template <bool FIRST, bool LAST>
__global__ void __launch_bounds__(kSortThreads)
    k_sort_pass(const int32_t* __restrict__ xyz, int n, int bits, int cap, int pass, int tiles,
                const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                uint32_t* __restrict__ lookback, int32_t* __restrict__ perm,
                uint32_t* __restrict__ pk, int32_t* __restrict__ rank1,
                int32_t* __restrict__ rank2, DevScalars* __restrict__ sc) {
  constexpr int kWarps = kSortThreads / 32;
  static_assert(kSortThreads == kRadix, "one thread per digit");
  __shared__ uint32_t s_whist[kWarps][kRadix];
  __shared__ uint32_t s_keys[kSortTile];
  __shared__ uint32_t s_vals[kSortTile];
  __shared__ uint32_t s_tstart[kRadix];
  __shared__ uint32_t s_gbase[kRadix];
  __shared__ uint32_t s_warp[kWarps];
  __shared__ int s_tile;
  __shared__ uint32_t s_count;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int shift = kRadixBits * pass;
  if (tid == 0) s_tile = int(atomicAdd(&sc->tile_counter[pass], 1u));
  for (int i = tid; i < kWarps * kRadix; i += kSortThreads) (&s_whist[0][0])[i] = 0;
  __syncthreads();
  const int tile_id = s_tile;
  const int code = tile_id / tiles;
  const int t = tile_id - code * tiles;
  const int warp_base = t * kSortTile + warp * (32 * kSortKpt);
  const size_t coff = size_t(code) * size_t(cap);

  uint32_t key[kSortKpt], val[kSortKpt], rnk[kSortKpt];
  const uint32_t m = (1u << bits) - 1u;
#pragma unroll
  for (int j = 0; j < kSortKpt; ++j) {
    const int pos = warp_base + j * 32 + lane;
    key[j] = 0;
    val[j] = 0;
    rnk[j] = 0;
    if (pos < n) {
      if (FIRST) {
        const uint32_t x = uint32_t(xyz[3 * size_t(pos)]) & m;
        const uint32_t y = uint32_t(xyz[3 * size_t(pos) + 1]) & m;
        const uint32_t z = uint32_t(xyz[3 * size_t(pos) + 2]) & m;
        key[j] = code_of(code, x, y, z, bits);
        val[j] = uint32_t(pos);
      } else {
        key[j] = keys_in[coff + pos];
        val[j] = vals_in[coff + pos];
      }
    }
  }

  // stable rank of each key among equal digits of its warp, in input order
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < kSortKpt; ++j) {
    const bool valid = (warp_base + j * 32 + lane) < n;
    const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
    const uint32_t d = (key[j] >> shift) & (kRadix - 1);
    uint32_t peers = 0, before = 0;
    if (valid) {
      peers = __match_any_sync(vmask, d);
      before = s_whist[warp][d];
    }
    __syncwarp();
    if (valid) {
      rnk[j] = before + __popc(peers & lt);
      if ((peers & lt) == 0) s_whist[warp][d] = before + __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();

  // per digit: offsets of the warps and the tile total
  const int d = tid;
  uint32_t total = 0;
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    const uint32_t c = s_whist[w][d];
    s_whist[w][d] = total;
    total += c;
  }
  const uint32_t tstart = block_exclusive_scan_256(total, s_warp);
  s_tstart[d] = tstart;
  if (d == kRadix - 1) s_count = tstart + total;
  const uint32_t gcount = sc->hist[code][pass][d];
  const uint32_t bstart = block_exclusive_scan_256(gcount, s_warp);

  // decoupled look-back over the earlier tiles of this code
  uint32_t* lb = lookback + size_t(code) * size_t(tiles) * kRadix;
  uint32_t prefix = 0;
  if (t == 0) {
    st_relaxed_gpu(&lb[d], kLbPre | total);
  } else {
    st_relaxed_gpu(&lb[size_t(t) * kRadix + d], kLbAgg | total);
    int p = t - 1;
    unsigned long long t0 = 0;
    while (true) {
      const uint32_t v = ld_relaxed_gpu(&lb[size_t(p) * kRadix + d]);
      const uint32_t f = v & kLbFlags;
      if (f == 0) {
        const unsigned long long now = global_ns();
        if (t0 == 0) t0 = now;
        if (now - t0 > kWaitLimitNs) {
          atomicOr(&sc->status, kFlagTimeout);
          break;
        }
        __nanosleep(32);
        continue;
      }
      prefix += v & kLbCount;
      if (f == kLbPre || p == 0) break;
      --p;
    }
    st_relaxed_gpu(&lb[size_t(t) * kRadix + d], kLbPre | ((prefix + total) & kLbCount));
  }
  s_gbase[d] = bstart + prefix;
  __syncthreads();

  // local sort of the tile by digit, then write out in digit runs
#pragma unroll
  for (int j = 0; j < kSortKpt; ++j) {
    if ((warp_base + j * 32 + lane) < n) {
      const uint32_t dj = (key[j] >> shift) & (kRadix - 1);
      const uint32_t lp = s_tstart[dj] + s_whist[warp][dj] + rnk[j];
      s_keys[lp] = key[j];
      s_vals[lp] = val[j];
    }
  }
  __syncthreads();
  const uint32_t cnt = s_count;
  for (uint32_t i = tid; i < cnt; i += kSortThreads) {
    const uint32_t k = s_keys[i], v = s_vals[i];
    const uint32_t dk = (k >> shift) & (kRadix - 1);
    const uint32_t g = s_gbase[dk] + (i - s_tstart[dk]);
    if (g >= uint32_t(n) || v >= uint32_t(n)) continue;  // only after a timed-out look-back
    if (!LAST) {
      keys_out[coff + g] = k;
      vals_out[coff + g] = v;
    } else {
      perm[coff + g] = int32_t(v);
      if (code == 0) {
        pk[g] = k;
        rank1[v] = int32_t(g);
      } else if (code == 1) {
        rank2[v] = int32_t(g);
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_link(int n, int bits, int cap, const int32_t* __restrict__ perm,
                                              const int32_t* __restrict__ rank1,
                                              const int32_t* __restrict__ rank2,
                                              const uint32_t* __restrict__ pk, int4* __restrict__ c4,
                                              DevScalars* __restrict__ sc) {
  __shared__ unsigned long long s_red[8];
  const int code = blockIdx.y;
  unsigned long long edges = 0, dist = 0;
  const float dscale = float(1u << kDistShift);
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    if (code == 0) {
      if (r + 1 < n) {
        const int d2 = sq_dist_c1(pk[r], pk[r + 1], bits);
        edges += 1;
        dist += (unsigned long long)__float2ull_rn(sqrtf(float(d2)) * dscale);
      }
      continue;
    }
    const int32_t* pc = perm + size_t(code) * size_t(cap);
    const int i = pc[r];
    if (!in_range(i, n)) continue;
    const int k = rank1[i];
    if (!in_range(k, n)) continue;
    int kp = -1, kn = -1;
    if (r > 0 && in_range(pc[r - 1], n)) {
      const int ip = pc[r - 1];
      const int kk = rank1[ip];
      bool dup = abs(k - kk) == 1;
      if (code == 2) dup |= abs(rank2[i] - rank2[ip]) == 1;
      kp = (dup || !in_range(kk, n)) ? -1 : kk;
    }
    if (r + 1 < n && in_range(pc[r + 1], n)) {
      const int in = pc[r + 1];
      const int kk = rank1[in];
      bool dup = abs(k - kk) == 1;
      if (code == 2) dup |= abs(rank2[i] - rank2[in]) == 1;
      if (!dup && in_range(kk, n)) {
        kn = kk;
        const int d2 = sq_dist_c1(pk[k], pk[kk], bits);
        edges += 1;
        dist += (unsigned long long)__float2ull_rn(sqrtf(float(d2)) * dscale);
      }
    }
    int2* slot = reinterpret_cast<int2*>(c4 + k) + (code - 1);
    *slot = make_int2(kp, kn);
  }
  edges = block_sum_u64<256>(edges, s_red);
  dist = block_sum_u64<256>(dist, s_red);
  if (threadIdx.x == 0) {
    if (edges) atomicAdd(&sc->n_edges, edges);
    if (dist) atomicAdd(&sc->dist_fx, dist);
  }
}

}  // namespace

cudaError_t launch_hist(const int32_t* xyz, int n, int bits, int passes, uint32_t* zero_buf,
                        size_t zero_words, DevScalars* sc, int num_sms, cudaStream_t stream) {
  const size_t work = std::max<size_t>(size_t(n), zero_words);
  int grid = int(std::min<size_t>((work + 2047) / 2048, size_t(num_sms) * 4));
  grid = std::max(grid, 1);
  k_hist<<<grid, 256, 0, stream>>>(xyz, n, bits, passes, zero_buf, zero_words, sc);
  return cudaGetLastError();
}

cudaError_t launch_sort_pass(int pass, int passes, const int32_t* xyz, int n, int bits, int cap,
                             const SortBufs& sb, const GraphBufs& gb, DevScalars* sc,
                             cudaStream_t stream) {
  const bool first = pass == 0, last = pass == passes - 1;
  const uint32_t* kin = first ? nullptr : sb.keys[(pass - 1) & 1];
  const uint32_t* vin = first ? nullptr : sb.vals[(pass - 1) & 1];
  uint32_t* kout = sb.keys[pass & 1];
  uint32_t* vout = sb.vals[pass & 1];
  uint32_t* lb = sb.lookback + size_t(pass) * 3 * size_t(sb.tiles) * kRadix;
  const dim3 grid(3 * sb.tiles);
#define FGBD_SORT_LAUNCH(F, L)                                                                    \
  k_sort_pass<F, L><<<grid, kSortThreads, 0, stream>>>(xyz, n, bits, cap, pass, sb.tiles, kin, vin, \
                                                       kout, vout, lb, gb.perm, gb.pk, gb.rank1,  \
                                                       gb.rank2, sc)
  if (first && last) FGBD_SORT_LAUNCH(true, true);
  else if (first) FGBD_SORT_LAUNCH(true, false);
  else if (last) FGBD_SORT_LAUNCH(false, true);
  else FGBD_SORT_LAUNCH(false, false);
#undef FGBD_SORT_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_link(int n, int bits, int cap, const GraphBufs& gb, DevScalars* sc, int num_sms,
                        cudaStream_t stream) {
  const int gx = std::max(1, std::min((n + 255) / 256, num_sms * 8));
  k_link<<<dim3(gx, 3), 256, 0, stream>>>(n, bits, cap, gb.perm, gb.rank1, gb.rank2, gb.pk, gb.c4, sc);
  return cudaGetLastError();
}

}  // namespace fgbd
