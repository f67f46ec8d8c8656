// SLG: scan-line graph construction (Section 2.2).
//
// 1. k_hist: scan-line codes C1..C3 (Eq. 1-3) of every point and the digit
//    histograms of every radix pass of every code, in one read of xyz.
// 2. one least-significant-digit pass of a stable radix sort over all three
//    codes at once (8-bit digits, 4096-key tiles), as reduce-then-scan:
//    k_tile_counts (digit counts per tile), k_tile_scan (each tile's start of
//    every digit) and k_sort_scatter (stable in-tile rank, write-out in digit
//    runs).  Ties keep input order, so equal codes are ordered by index.  The
//    last pass writes the orders, the packed C1 code of each sorted point, and
//    the C1/C2 rank of each input point.
// 3. k_link: points consecutive along a code are linked (Section 2.2).  In C1
//    order the code-1 neighbours are implicit (k-1, k+1); C2/C3 neighbours
//    are written as slots, a pair already linked by an earlier code is left
//    out so the union is a set, and each distinct edge's length is summed
//    for sigma_g.
#include <algorithm>

#include "fgbd_internal.cuh"

namespace fgbd {
namespace {



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

// The keys of tile t of code c at this pass (striped: item j of lane l of warp
// w is position t*kSortTile + w*32*kSortKpt + j*32 + l, so loads coalesce).
template <bool FIRST>
__device__ __forceinline__ void load_tile(const int32_t* __restrict__ xyz, const uint32_t* __restrict__ keys_in,
                                          const uint32_t* __restrict__ vals_in, int n, int bits, size_t coff,
                                          int code, int warp_base, int lane, uint32_t (&key)[kSortKpt],
                                          uint32_t (&val)[kSortKpt], bool with_vals) {
  const uint32_t m = (1u << bits) - 1u;
#pragma unroll
  for (int j = 0; j < kSortKpt; ++j) {
    const int pos = warp_base + j * 32 + lane;
    key[j] = 0;
    val[j] = 0;
    if (pos < n) {
      if (FIRST) {
        const uint32_t x = uint32_t(xyz[3 * size_t(pos)]) & m;
        const uint32_t y = uint32_t(xyz[3 * size_t(pos) + 1]) & m;
        const uint32_t z = uint32_t(xyz[3 * size_t(pos) + 2]) & m;
        key[j] = code_of(code, x, y, z, bits);
        val[j] = uint32_t(pos);
      } else {
        key[j] = keys_in[coff + pos];
        if (with_vals) val[j] = vals_in[coff + pos];
      }
    }
  }
}

// Reduce: digit counts of every tile, counts[(code*kRadix + digit)*tiles + tile].
template <bool FIRST>
__global__ void __launch_bounds__(kSortThreads)
    k_tile_counts(const int32_t* __restrict__ xyz, int n, int bits, int cap, int pass, int tiles,
                  const uint32_t* __restrict__ keys_in, uint32_t* __restrict__ counts) {
  __shared__ uint32_t s_h[kRadix];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int code = blockIdx.x / tiles;
  const int t = blockIdx.x - code * tiles;
  s_h[tid] = 0;
  __syncthreads();
  uint32_t key[kSortKpt], val[kSortKpt];
  load_tile<FIRST>(xyz, keys_in, nullptr, n, bits, size_t(code) * size_t(cap), code,
                   t * kSortTile + warp * (32 * kSortKpt), lane, key, val, false);
  const int shift = kRadixBits * pass;
#pragma unroll
  for (int j = 0; j < kSortKpt; ++j)
    if (t * kSortTile + warp * (32 * kSortKpt) + j * 32 + lane < n) atomicAdd(&s_h[(key[j] >> shift) & (kRadix - 1)], 1u);
  __syncthreads();
  counts[(size_t(code) * kRadix + tid) * tiles + t] = s_h[tid];
}

// Scan: one warp per (code, digit) row.  offsets[row][t] = start of the
// digit's bucket (sum of the smaller digits' totals) + counts of tiles < t.
__global__ void __launch_bounds__(256) k_tile_scan(int tiles, int pass, const DevScalars* __restrict__ sc,
                                                   uint32_t* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  const int row = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (row >= 3 * kRadix) return;
  const int code = row / kRadix, d = row - code * kRadix;
  uint32_t base = 0;
  for (int e = lane; e < d; e += 32) base += sc->hist[code][pass][e];
  base = warp_sum(base);
  uint32_t* r = counts + size_t(row) * tiles;
  for (int t0 = 0; t0 < tiles; t0 += 32) {
    const int t = t0 + lane;
    const uint32_t c = t < tiles ? r[t] : 0u;
    uint32_t x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (t < tiles) r[t] = base + x - c;
    base += __shfl_sync(0xffffffffu, x, 31);
  }
}

// Scatter: rank each key of the tile among equal digits (stable), then write
// the tile out in digit runs at the offsets the scan produced.  The last pass
// writes the orders, the packed C1 codes and the C1/C2 ranks instead.
template <bool FIRST, bool LAST>
__global__ void __launch_bounds__(kSortThreads, 3)
    k_sort_scatter(const int32_t* __restrict__ xyz, int n, int bits, int cap, int pass, int tiles,
                   const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                   uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                   const uint32_t* __restrict__ offsets, int32_t* __restrict__ perm, uint32_t* __restrict__ pk,
                   int32_t* __restrict__ rank1, int32_t* __restrict__ rank2) {
  constexpr int kWarps = kSortThreads / 32;
  static_assert(kSortThreads == kRadix, "one thread per digit");
  __shared__ uint32_t s_whist[kWarps][kRadix];
  __shared__ uint32_t s_keys[kSortTile];
  __shared__ uint32_t s_vals[kSortTile];
  __shared__ uint32_t s_tstart[kRadix];
  __shared__ uint32_t s_gbase[kRadix];
  __shared__ uint32_t s_warp[kWarps];
  __shared__ uint32_t s_count;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int shift = kRadixBits * pass;
  for (int i = tid; i < kWarps * kRadix; i += kSortThreads) (&s_whist[0][0])[i] = 0;
  const int code = blockIdx.x / tiles;
  const int t = blockIdx.x - code * tiles;
  const int warp_base = t * kSortTile + warp * (32 * kSortKpt);
  const size_t coff = size_t(code) * size_t(cap);
  // this tile's global start of every digit, known before any key is ranked
  const uint32_t gbase = offsets[(size_t(code) * kRadix + tid) * tiles + t];

  uint32_t key[kSortKpt], val[kSortKpt], rnk[kSortKpt];
  load_tile<FIRST>(xyz, keys_in, vals_in, n, bits, coff, code, warp_base, lane, key, val, true);
  __syncthreads();

  // stable rank of each key among equal digits of its warp, in input order:
  // the lanes with the same digit are found with one ballot per digit bit; the
  // lowest of them adds the group size to the warp's digit counter and the
  // count it returns is the group's base
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < kSortKpt; ++j) {
    const bool valid = (warp_base + j * 32 + lane) < n;
    const uint32_t d = (key[j] >> shift) & (kRadix - 1);
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int b = 0; b < kRadixBits; ++b) {
      const bool bit = (d >> b) & 1u;
      const uint32_t on = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? on : ~on;
    }
    const int leader = peers ? __ffs(peers) - 1 : lane;
    uint32_t old = 0;
    if (valid && lane == leader) old = atomicAdd(&s_whist[warp][d], uint32_t(__popc(peers)));
    rnk[j] = __shfl_sync(0xffffffffu, old, leader) + __popc(peers & lt);
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
  s_gbase[d] = gbase;
  if (d == kRadix - 1) s_count = tstart + total;
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
    if (g >= uint32_t(n) || v >= uint32_t(n)) continue;
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

// One thread per position r of one code's order (blockIdx.y = code).  Each
// thread resolves its own point only (input index, sorted id, C2 rank and
// packed code); the values at positions r-1 and r+1 come from the adjacent
// lanes, with one extra lookup at each end of the warp.
struct LinkPt {
  int k;       // sorted (C1) id, -1 outside [0, n)
  int r2;      // position in the C2 order (code 2 only)
  uint32_t c;  // packed C1 code
};

__device__ __forceinline__ LinkPt link_point(int r, int n, int code, const int32_t* __restrict__ pc,
                                             const int32_t* __restrict__ rank1, const int32_t* __restrict__ rank2,
                                             const uint32_t* __restrict__ pk) {
  LinkPt q{-1, -1, 0u};
  if (r < 0 || r >= n) return q;
  if (code == 0) {
    q.k = r;
    q.c = pk[r];
    return q;
  }
  const int i = pc[r];
  if (!in_range(i, n)) return q;
  const int k = rank1[i];
  if (!in_range(k, n)) return q;
  q.k = k;
  q.c = pk[k];
  if (code == 2) q.r2 = rank2[i];
  return q;
}

__global__ void __launch_bounds__(256) k_link(int n, int bits, int cap, const int32_t* __restrict__ perm,
                                              const int32_t* __restrict__ rank1,
                                              const int32_t* __restrict__ rank2,
                                              const uint32_t* __restrict__ pk, int4* __restrict__ c4,
                                              DevScalars* __restrict__ sc) {
  __shared__ unsigned long long s_red[8];
  const int code = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int32_t* pc = perm + size_t(code) * size_t(cap);
  unsigned long long edges = 0;
  float dist_f = 0.f;  // this thread's few edge lengths; converted to fixed point once
  const int stride = gridDim.x * blockDim.x;
  // whole warps step together so the shuffles see every lane
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int r = base + lane;
    const LinkPt me = link_point(r, n, code, pc, rank1, rank2, pk);
    LinkPt prev, next;
    prev.k = __shfl_up_sync(0xffffffffu, me.k, 1);
    prev.r2 = __shfl_up_sync(0xffffffffu, me.r2, 1);
    prev.c = __shfl_up_sync(0xffffffffu, me.c, 1);
    next.k = __shfl_down_sync(0xffffffffu, me.k, 1);
    next.r2 = __shfl_down_sync(0xffffffffu, me.r2, 1);
    next.c = __shfl_down_sync(0xffffffffu, me.c, 1);
    if (lane == 0) prev = link_point(r - 1, n, code, pc, rank1, rank2, pk);
    if (lane == 31) next = link_point(r + 1, n, code, pc, rank1, rank2, pk);
    if (me.k < 0) continue;
    // the edge to the next position: counted once, unless an earlier code links the pair
    bool dup_next = true;
    if (next.k >= 0) {
      dup_next = code > 0 && abs(me.k - next.k) == 1;
      if (code == 2) dup_next |= abs(me.r2 - next.r2) == 1;
      if (!dup_next) {
        edges += 1;
        dist_f += sqrtf(float(sq_dist_c1(me.c, next.c, bits)));
      }
    }
    if (code == 0) continue;
    bool dup_prev = true;
    if (prev.k >= 0) {
      dup_prev = abs(me.k - prev.k) == 1;
      if (code == 2) dup_prev |= abs(me.r2 - prev.r2) == 1;
    }
    int2* slot = reinterpret_cast<int2*>(c4 + me.k) + (code - 1);
    *slot = make_int2(dup_prev ? -1 : prev.k, dup_next ? -1 : next.k);
  }
  unsigned long long dist = (unsigned long long)__float2ull_rn(dist_f * float(1u << kDistShift));
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
  uint32_t* counts = sb.tile_counts + size_t(pass) * 3 * size_t(sb.tiles) * kRadix;
  const dim3 grid(3 * sb.tiles);
  if (first) k_tile_counts<true><<<grid, kSortThreads, 0, stream>>>(xyz, n, bits, cap, pass, sb.tiles, kin, counts);
  else k_tile_counts<false><<<grid, kSortThreads, 0, stream>>>(xyz, n, bits, cap, pass, sb.tiles, kin, counts);
  k_tile_scan<<<(3 * kRadix + 7) / 8, 256, 0, stream>>>(sb.tiles, pass, sc, counts);
#define FGBD_SCATTER(F, L)                                                                              \
  k_sort_scatter<F, L><<<grid, kSortThreads, 0, stream>>>(xyz, n, bits, cap, pass, sb.tiles, kin, vin, kout, vout, \
                                                          counts, gb.perm, gb.pk, gb.rank1, gb.rank2)
  if (first && last) FGBD_SCATTER(true, true);
  else if (first) FGBD_SCATTER(true, false);
  else if (last) FGBD_SCATTER(false, true);
  else FGBD_SCATTER(false, false);
#undef FGBD_SCATTER
  return cudaGetLastError();
}

cudaError_t launch_link(int n, int bits, int cap, const GraphBufs& gb, DevScalars* sc, int num_sms,
                        cudaStream_t stream) {
  const int gx = std::max(1, std::min((n + 255) / 256, num_sms * 8));
  k_link<<<dim3(gx, 3), 256, 0, stream>>>(n, bits, cap, gb.perm, gb.rank1, gb.rank2, gb.pk, gb.c4, sc);
  return cudaGetLastError();
}

}  // namespace fgbd
