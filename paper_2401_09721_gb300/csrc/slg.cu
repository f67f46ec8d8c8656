// SLG: scan-line graph construction (Section 2.2).
//
// Sorting by a code of Eq. 1-3 is sorting by three b-bit coordinates, most
// significant first, so a least-significant-digit radix sort whose digits are
// the coordinates needs three passes of 2^b bins:
//   C1 = (z, y, x): passes on x, then y, then z, from the input order;
//   C2 = (x, z, y): one stable pass on x over the C1 order (among points
//        with equal x the C1 order already ranks them by (z, y));
//   C3 = (y, x, z): one stable pass on y over the C2 order (among points
//        with equal y the C2 order ranks them by (x, z)).
// Ties keep input order throughout, so equal codes are ordered by index.  The
// digit totals of every pass are the three coordinate histograms, taken once
// (k_coord_hist).  Each pass is reduce-then-scan:
//   k_tile_counts   digit counts of every 4096-key tile;
//   k_tile_scan     each tile's global start of every digit;
//   k_sort_scatter  stable in-tile rank (one ballot per digit bit) and
//                   write-out in digit runs.
// The C1 passes carry (code, input index) and end with the packed C1 code of
// every sorted point, its input index and the rank of every input point; the
// C2/C3 passes carry (code, sorted id) and end with the sorted ids along C2
// and C3 and the C2 rank of every sorted id.
// k_link: points consecutive along a code are linked.  In C1 order the code-1
// neighbours are implicit (k-1, k+1); C2/C3 neighbours are written as slots;
// a pair already linked by an earlier code is left out so the union is a set,
// and each distinct edge's length is summed for sigma_g.
#include <algorithm>

#include "fgbd_internal.cuh"

namespace fgbd {
namespace {

// The scatter runs 512 threads on a 4096-key tile (8 keys a thread), twice
// the threads of the counting pass, so that the per-block serial chains
// (ranking, write-out) are half as long.  Two warps share one 32-bit digit
// counter word (16 bits each: a warp ranks at most 256 keys).
constexpr int kScatterThreads = 512;
constexpr int kScatterWarps = kScatterThreads / 32;         // 16
constexpr int kScatterKpt = kSortTile / kScatterThreads;     // 8
constexpr int kPairWords = kScatterWarps / 2;               // counter words per digit
constexpr int kDigitsPerThread = kMaxRadix / kScatterThreads;  // 2

size_t scatter_smem_bytes() {
  return sizeof(uint32_t) *
         (size_t(kPairWords) * kMaxRadix + 2 * size_t(kSortTile) + 2 * size_t(kMaxRadix) + kScatterWarps + 1);
}

__global__ void __launch_bounds__(256) k_coord_hist(const int32_t* __restrict__ xyz, int n, int bits,
                                                    DevScalars* __restrict__ sc) {
  __shared__ uint32_t h[3][kMaxRadix];
  const int radix = 1 << bits;
  for (int i = threadIdx.x; i < 3 * kMaxRadix; i += blockDim.x) (&h[0][0])[i] = 0;
  __syncthreads();
  const uint32_t m = uint32_t(radix) - 1u;
  bool bad = false;
  const size_t gstride = size_t(gridDim.x) * blockDim.x;
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < size_t(n); i += gstride) {
    const int xi = xyz[3 * i], yi = xyz[3 * i + 1], zi = xyz[3 * i + 2];
    bad |= (uint32_t(xi) > m) | (uint32_t(yi) > m) | (uint32_t(zi) > m);
    atomicAdd(&h[0][uint32_t(xi) & m], 1u);
    atomicAdd(&h[1][uint32_t(yi) & m], 1u);
    atomicAdd(&h[2][uint32_t(zi) & m], 1u);
  }
  if (bad) atomicOr(&sc->status, kFlagRange);
  __syncthreads();
  for (int c = 0; c < 3; ++c)
    for (int d = threadIdx.x; d < radix; d += blockDim.x)
      if (h[c][d]) atomicAdd(&sc->chist[c][d], h[c][d]);
}

// The keys and values of one tile (striped: item j of lane l of warp w is
// position t*kSortTile + w*32*kSortKpt + j*32 + l, so loads coalesce).
__device__ __forceinline__ void load_tile(const SortPassArgs& a, int warp_base, int lane, uint32_t (&key)[kSortKpt],
                                          uint32_t (&val)[kSortKpt], bool with_vals) {
  const uint32_t m = (1u << a.bits) - 1u;
#pragma unroll
  for (int j = 0; j < kSortKpt; ++j) {
    const int pos = warp_base + j * 32 + lane;
    key[j] = 0;
    val[j] = 0;
    if (pos < a.n) {
      if (a.xyz) {
        const uint32_t x = uint32_t(a.xyz[3 * size_t(pos)]) & m;
        const uint32_t y = uint32_t(a.xyz[3 * size_t(pos) + 1]) & m;
        const uint32_t z = uint32_t(a.xyz[3 * size_t(pos) + 2]) & m;
        key[j] = code_of(0, x, y, z, a.bits);
        val[j] = uint32_t(pos);
      } else {
        key[j] = a.keys_in[pos];
        if (with_vals) val[j] = a.vals_in ? a.vals_in[pos] : uint32_t(pos);
      }
    }
  }
}

// Reduce: digit counts of every tile, counts[digit * tiles + tile].
__global__ void __launch_bounds__(kSortThreads) k_tile_counts(SortPassArgs a) {
  __shared__ uint32_t s_h[kMaxRadix];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int radix = 1 << a.bits;
  const int t = blockIdx.x;
  for (int d = tid; d < radix; d += kSortThreads) s_h[d] = 0;
  __syncthreads();
  uint32_t key[kSortKpt], val[kSortKpt];
  const int warp_base = t * kSortTile + warp * (32 * kSortKpt);
  load_tile(a, warp_base, lane, key, val, false);
  const uint32_t m = uint32_t(radix) - 1u;
#pragma unroll
  for (int j = 0; j < kSortKpt; ++j)
    if (warp_base + j * 32 + lane < a.n) atomicAdd(&s_h[(key[j] >> a.shift) & m], 1u);
  __syncthreads();
  for (int d = tid; d < radix; d += kSortThreads) a.counts[size_t(d) * a.tiles + t] = s_h[d];
}

// Scan: one warp per digit row.  counts become offsets: the start of the
// digit's bucket (total of the smaller digits) plus the counts of the earlier
// tiles.  Each lane owns a run of up to 8 consecutive tiles per batch.
__global__ void __launch_bounds__(256) k_tile_scan(SortPassArgs a) {
  const int lane = threadIdx.x & 31;
  const int radix = 1 << a.bits;
  const int d = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (d >= radix) return;
  // the digit's bucket start: lane l sums the histogram entries 32l..32l+31
  // below d, read as eight independent 16-byte loads
  const uint4* hist4 = reinterpret_cast<const uint4*>(a.sc->chist[a.coord]);
  uint32_t base = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int e = lane * 32 + i * 4;
    if (e < d) {
      const uint4 h = hist4[e >> 2];
      base += h.x + (e + 1 < d ? h.y : 0u) + (e + 2 < d ? h.z : 0u) + (e + 3 < d ? h.w : 0u);
    }
  }
  base = warp_sum(base);
  uint32_t* r = a.counts + size_t(d) * a.tiles;
  constexpr int kRun = 8;
  for (int t0 = 0; t0 < a.tiles; t0 += 32 * kRun) {
    uint32_t c[kRun];
    uint32_t own = 0;
#pragma unroll
    for (int i = 0; i < kRun; ++i) {
      const int t = t0 + lane * kRun + i;
      c[i] = t < a.tiles ? r[t] : 0u;
      own += c[i];
    }
    uint32_t x = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    uint32_t run = base + x - own;
#pragma unroll
    for (int i = 0; i < kRun; ++i) {
      const int t = t0 + lane * kRun + i;
      if (t < a.tiles) r[t] = run;
      run += c[i];
    }
    base += __shfl_sync(0xffffffffu, x, 31);
  }
}

// Scatter: rank each key of the tile among equal digits (stable), then write
// the tile out in digit runs at the offsets the scan produced.
__global__ void __launch_bounds__(kScatterThreads, 2) k_sort_scatter(SortPassArgs a) {
  extern __shared__ uint32_t smem[];
  uint32_t* s_whist = smem;                             // [kPairWords][radix]: warps 2w, 2w+1 in the low, high half
  uint32_t* s_keys = s_whist + kPairWords * kMaxRadix;  // [kSortTile]
  uint32_t* s_vals = s_keys + kSortTile;                // [kSortTile]
  uint32_t* s_tstart = s_vals + kSortTile;              // [radix]
  uint32_t* s_gbase = s_tstart + kMaxRadix;             // [radix]
  uint32_t* s_warp = s_gbase + kMaxRadix;               // [kScatterWarps]
  uint32_t* s_count = s_warp + kScatterWarps;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bits = a.bits, radix = 1 << bits;
  const uint32_t m = uint32_t(radix) - 1u;
  const int t = blockIdx.x;
  const int shift = a.shift;
  const int warp_base = t * kSortTile + warp * (32 * kScatterKpt);
  for (int i = tid; i < kPairWords * radix; i += kScatterThreads) s_whist[i] = 0;
  // this tile's global start of every digit, known before any key is ranked
  for (int d = tid; d < radix; d += kScatterThreads) s_gbase[d] = a.counts[size_t(d) * a.tiles + t];

  // the keys and values of this warp's 256 positions (striped, so loads coalesce)
  uint32_t key[kScatterKpt], val[kScatterKpt], rnk[kScatterKpt];
#pragma unroll
  for (int j = 0; j < kScatterKpt; ++j) {
    const int pos = warp_base + j * 32 + lane;
    key[j] = 0;
    val[j] = 0;
    if (pos < a.n) {
      if (a.xyz) {
        const uint32_t x = uint32_t(a.xyz[3 * size_t(pos)]) & m;
        const uint32_t y = uint32_t(a.xyz[3 * size_t(pos) + 1]) & m;
        const uint32_t z = uint32_t(a.xyz[3 * size_t(pos) + 2]) & m;
        key[j] = code_of(0, x, y, z, bits);
        val[j] = uint32_t(pos);
      } else {
        key[j] = a.keys_in[pos];
        val[j] = a.vals_in ? a.vals_in[pos] : uint32_t(pos);
      }
    }
  }
  __syncthreads();

  // stable rank of each key among equal digits of its warp, in input order:
  // the lanes with the same digit are found with one ballot per digit bit; the
  // lowest of them adds the group size to the warp's digit counter and the
  // count it gets back is the group's base
  uint32_t* wh = s_whist + (warp >> 1) * radix;
  const int half = 16 * (warp & 1);
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < kScatterKpt; ++j) {
    const bool valid = (warp_base + j * 32 + lane) < a.n;
    const uint32_t d = (key[j] >> shift) & m;
    uint32_t peers = __ballot_sync(0xffffffffu, valid);
    for (int b = 0; b < bits; ++b) {
      const bool bit = (d >> b) & 1u;
      const uint32_t on = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? on : ~on;
    }
    const int leader = peers ? __ffs(peers) - 1 : lane;
    uint32_t old = 0;
    if (valid && lane == leader) old = (atomicAdd(&wh[d], uint32_t(__popc(peers)) << half) >> half) & 0xffffu;
    rnk[j] = __shfl_sync(0xffffffffu, old, leader) + __popc(peers & lt);
    __syncwarp();
  }
  __syncthreads();

  // per digit (each thread owns kDigitsPerThread consecutive digits): offsets
  // of the warps, the tile total, and the tile's exclusive digit start
  uint32_t tot[kDigitsPerThread];
  uint32_t own = 0;
#pragma unroll
  for (int i = 0; i < kDigitsPerThread; ++i) {
    const int d = tid * kDigitsPerThread + i;
    uint32_t run = 0;
    if (d < radix) {
#pragma unroll
      for (int w = 0; w < kPairWords; ++w) {
        const uint32_t c = s_whist[w * radix + d];
        const uint32_t lo = c & 0xffffu, hi = c >> 16;
        s_whist[w * radix + d] = run | ((run + lo) << 16);
        run += lo + hi;
      }
    }
    tot[i] = run;
    own += run;
  }
  {
    uint32_t x = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    uint32_t off = 0;
#pragma unroll
    for (int w = 0; w < kScatterWarps; ++w) off += (w < warp) ? s_warp[w] : 0u;
    uint32_t start = off + x - own;
#pragma unroll
    for (int i = 0; i < kDigitsPerThread; ++i) {
      const int d = tid * kDigitsPerThread + i;
      if (d < radix) s_tstart[d] = start;
      start += tot[i];
    }
    if (tid == kScatterThreads - 1) *s_count = start;
  }
  __syncthreads();

  // local sort of the tile by digit, then write out in digit runs
#pragma unroll
  for (int j = 0; j < kScatterKpt; ++j) {
    if ((warp_base + j * 32 + lane) < a.n) {
      const uint32_t dj = (key[j] >> shift) & m;
      const uint32_t lp = s_tstart[dj] + ((wh[dj] >> half) & 0xffffu) + rnk[j];
      s_keys[lp] = key[j];
      s_vals[lp] = val[j];
    }
  }
  __syncthreads();
  const uint32_t cnt = *s_count;
  uint32_t* ko = a.keys_out;
  uint32_t* vo = a.vals_out;
  int32_t* ro = a.rank_out;
  for (uint32_t i = tid; i < cnt; i += kScatterThreads) {
    const uint32_t k = s_keys[i], v = s_vals[i];
    const uint32_t dk = (k >> shift) & m;
    const uint32_t g = s_gbase[dk] + (i - s_tstart[dk]);
    if (g >= uint32_t(a.n) || v >= uint32_t(a.n)) continue;
    if (ko) ko[g] = k;
    if (vo) vo[g] = v;
    if (ro) ro[v] = int32_t(g);
  }
}

// One thread per position r of one code's order (blockIdx.y = code).  Code 0
// is the C1 order itself; codes 1 and 2 read the sorted ids along C2 and C3.
// The ids at r-1 and r+1 come from the adjacent lanes, with one extra lookup
// at each end of the warp.
struct LinkPt {
  int k;       // sorted (C1) id, -1 outside [0, n)
  int r2;      // position in the C2 order (code 2 only)
  uint32_t c;  // packed C1 code
};

__device__ __forceinline__ LinkPt link_point(int r, int n, int code, const int32_t* __restrict__ ord,
                                             const int32_t* __restrict__ rank2, const uint32_t* __restrict__ pk) {
  LinkPt q{-1, -1, 0u};
  if (r < 0 || r >= n) return q;
  const int k = code == 0 ? r : ord[r];
  if (!in_range(k, n)) return q;
  q.k = k;
  q.c = pk[k];
  if (code == 2) q.r2 = rank2[k];
  return q;
}

__global__ void __launch_bounds__(256) k_link(int n, int bits, int cap, const int32_t* __restrict__ ord23,
                                              const int32_t* __restrict__ rank2, const uint32_t* __restrict__ pk,
                                              int4* __restrict__ c4, DevScalars* __restrict__ sc) {
  __shared__ unsigned long long s_red[8];
  const int code = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int32_t* ord = code == 0 ? nullptr : ord23 + size_t(code - 1) * size_t(cap);
  unsigned long long edges = 0;
  float dist_f = 0.f;  // this thread's few edge lengths; converted to fixed point once
  const int stride = gridDim.x * blockDim.x;
  // whole warps step together so the shuffles see every lane
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int r = base + lane;
    const LinkPt me = link_point(r, n, code, ord, rank2, pk);
    LinkPt prev, next;
    prev.k = __shfl_up_sync(0xffffffffu, me.k, 1);
    prev.r2 = __shfl_up_sync(0xffffffffu, me.r2, 1);
    prev.c = __shfl_up_sync(0xffffffffu, me.c, 1);
    next.k = __shfl_down_sync(0xffffffffu, me.k, 1);
    next.r2 = __shfl_down_sync(0xffffffffu, me.r2, 1);
    next.c = __shfl_down_sync(0xffffffffu, me.c, 1);
    if (lane == 0) prev = link_point(r - 1, n, code, ord, rank2, pk);
    if (lane == 31) next = link_point(r + 1, n, code, ord, rank2, pk);
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

// The three orders in input indices: C1 from perm1, C2 and C3 through perm1.
__global__ void __launch_bounds__(256) k_orders_export(int n, int cap, const int32_t* __restrict__ perm1,
                                                       const int32_t* __restrict__ ord23, int32_t* __restrict__ out) {
  const int stride = gridDim.x * blockDim.x;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    out[r] = perm1[r];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int k = ord23[size_t(c) * size_t(cap) + r];
      out[size_t(c + 1) * size_t(n) + r] = in_range(k, n) ? perm1[k] : -1;
    }
  }
}

}  // namespace

cudaError_t launch_coord_hist(const int32_t* xyz, int n, int bits, DevScalars* sc, int num_sms, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = std::max(1, std::min((n + 2047) / 2048, num_sms * 4));
  k_coord_hist<<<grid, 256, 0, stream>>>(xyz, n, bits, sc);
  return cudaGetLastError();
}

cudaError_t launch_tile_counts(const SortPassArgs& a, cudaStream_t stream) {
  k_tile_counts<<<dim3(a.tiles), kSortThreads, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_tile_scan(const SortPassArgs& a, cudaStream_t stream) {
  k_tile_scan<<<((1 << a.bits) + 7) / 8, 256, 0, stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sort_scatter(const SortPassArgs& a, cudaStream_t stream) {
  // the shared-memory limit is a per-device function attribute: set it once per device
  static unsigned long long configured = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(configured & bit)) {
    e = cudaFuncSetAttribute(k_sort_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, int(scatter_smem_bytes()));
    if (e != cudaSuccess) return e;
    configured |= bit;
  }
  k_sort_scatter<<<dim3(a.tiles), kScatterThreads, scatter_smem_bytes(), stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sort_pass(const SortPassArgs& a, cudaStream_t stream) {
  cudaError_t e = launch_tile_counts(a, stream);
  if (e == cudaSuccess) e = launch_tile_scan(a, stream);
  if (e == cudaSuccess) e = launch_sort_scatter(a, stream);
  return e;
}

cudaError_t launch_link(int n, int bits, int cap, const GraphBufs& gb, DevScalars* sc, int num_sms,
                        cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int gx = std::max(1, std::min((n + 255) / 256, num_sms * 8));
  k_link<<<dim3(gx, 3), 256, 0, stream>>>(n, bits, cap, gb.ord23, gb.rank2, gb.pk, gb.c4, sc);
  return cudaGetLastError();
}

cudaError_t launch_orders_export(int n, int cap, const GraphBufs& gb, int32_t* out, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = std::max(1, std::min((n + 255) / 256, 152 * 16));
  k_orders_export<<<grid, 256, 0, stream>>>(n, cap, gb.perm1, gb.ord23, out);
  return cudaGetLastError();
}

SortPassArgs slg_pass_args(int pass, const int32_t* xyz, int n, int bits, int cap, const SortBufs& sb,
                           const GraphBufs& gb, const DevScalars* sc) {
  SortPassArgs a{};
  a.n = n;
  a.bits = bits;
  a.tiles = (n + kSortTile - 1) / kSortTile;
  a.counts = sb.tile_counts;
  a.sc = sc;
  if (pass < 3) {
    // C1: digits x, y, z; keys are packed C1 codes (x lowest), values input indices
    a.shift = pass * bits;
    a.coord = pass;
    a.xyz = pass == 0 ? xyz : nullptr;
    a.keys_in = pass == 0 ? nullptr : sb.keys[(pass - 1) & 1];
    a.vals_in = pass == 0 ? nullptr : sb.vals[(pass - 1) & 1];
    const bool last = pass == 2;
    a.keys_out = last ? gb.pk : sb.keys[pass & 1];
    a.vals_out = last ? reinterpret_cast<uint32_t*>(gb.perm1) : sb.vals[pass & 1];
    a.rank_out = last ? gb.rank1 : nullptr;
    return a;
  }
  if (pass == 3) {
    // C2: the C1 order (value = position = sorted id) on x
    a.shift = 0;
    a.coord = 0;
    a.keys_in = gb.pk;
    a.vals_in = nullptr;
    a.keys_out = sb.keys[0];
    a.vals_out = reinterpret_cast<uint32_t*>(gb.ord23);
    a.rank_out = gb.rank2;
    return a;
  }
  // C3: the C2 order on y
  a.shift = bits;
  a.coord = 1;
  a.keys_in = sb.keys[0];
  a.vals_in = reinterpret_cast<const uint32_t*>(gb.ord23);
  a.keys_out = nullptr;
  a.vals_out = reinterpret_cast<uint32_t*>(gb.ord23 + size_t(cap));
  a.rank_out = nullptr;
  return a;
}

}  // namespace fgbd
