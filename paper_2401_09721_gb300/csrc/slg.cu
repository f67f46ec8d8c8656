// SLG: scan-line graph construction (Section 2.2).
//
// Sorting by a code of Eq. 1-3 is sorting by three b-bit coordinates, most
// significant first.  The digits of the radix passes are the coordinates
// themselves (2^b bins), and ties keep input order throughout, so equal codes
// are ordered by index:
//   pass 0   one stable pass on y over the input puts every y-slab in place;
//   slab     k_slab_sort sorts each y-slab by (x, z) in shared memory, one
//            block per slab (two stable passes, z then x): the C3 = (y, x, z)
//            order;
//   pass 1   C1 = (z, y, x): one stable pass on z over the C3 order (among
//            points with equal z the C3 order already ranks them by (y, x));
//   pass 2   C2 = (x, z, y): one stable pass on x over the C1 order (among
//            points with equal x the C1 order ranks them by (z, y)).
// The digit totals of every pass are the three coordinate histograms, taken
// once (k_coord_hist).  Each global pass is reduce-then-scan:
//   k_tile_counts   digit counts of every 4096-key tile;
//   k_tile_scan     each tile's global start of every digit;
//   k_sort_scatter  stable in-tile rank (one ballot per digit bit) and
//                   write-out in digit runs.
// Keys are the packed C1 codes in every pass.  Pass 1 ends with the packed
// code of every sorted (C1) point, its input index, the rank of every input
// point, and the C3 order rewritten as sorted ids; pass 2 ends with the sorted
// ids along C2, their packed codes, and the C2 rank of every sorted id.
// k_link: points consecutive along a code are linked.  In C1 order the code-1
// neighbours are implicit (k-1, k+1); C2/C3 neighbours are written as slots;
// a pair already linked by an earlier code is left out so the union is a set,
// and each distinct edge's length is summed for sigma_g.
#include <algorithm>
#include <cstdlib>

#include "fgbd_internal.cuh"

namespace fgbd {
namespace {

// The scatter ranks a 4096-key tile with THREADS threads (the one-frame path
// runs 512, twice the threads of the counting pass, so that the per-block
// serial chains - ranking, write-out - are half as long; the batch tuner may
// pick 256 or 1024).  Two warps share one 32-bit digit counter word (16 bits
// each: a warp ranks at most 512 keys).
template <int THREADS>
struct ScatterShape {
  static constexpr int kWarps = THREADS / 32;
  static constexpr int kKpt = kSortTile / THREADS;          // keys per thread
  static constexpr int kPairWords = kWarps / 2;             // counter words per digit
  static constexpr int kDigitsPerThread = kMaxRadix / THREADS;
  static constexpr int kMinBlocks = THREADS >= 1024 ? 1 : 2;
  static_assert(kSortTile % THREADS == 0 && kMaxRadix % THREADS == 0 && kWarps % 2 == 0 && 32 * kKpt <= 65535,
                "tile, digits and counter halves must divide evenly");
};
constexpr int kScatterThreads = 512;  // the one-frame path

size_t scatter_smem_bytes(int threads) {
  const int warps = threads / 32;
  return sizeof(uint32_t) *
         (size_t(warps / 2) * kMaxRadix + 2 * size_t(kSortTile) + 2 * size_t(kMaxRadix) + warps + 1);
}

// The three coordinate histograms, 1024-thread blocks (up to two per SM) taking
// whole 4096-point tiles of the input, merged with global atomics.  The y digits of
// each tile are also counted on their own: sort pass 0's tile counts (its
// keys are the input's y digits in input order), so that pass needs no
// counting launch.  Pass 1's tile counts, which the slab sort adds up, are
// zeroed here.
__device__ __forceinline__ void coord_hist_body(const HistArgs& a, int bid, int nblk) {
  __shared__ uint32_t h[3][kMaxRadix];
  __shared__ uint32_t ht[kMaxRadix];
  const int radix = 1 << a.bits;
  const int tiles = (a.n + kSortTile - 1) / kSortTile;
  for (int i = threadIdx.x; i < 3 * kMaxRadix; i += blockDim.x) (&h[0][0])[i] = 0;
  if (a.counts1) {
    const size_t words = size_t(radix) * tiles;
    for (size_t i = size_t(bid) * blockDim.x + threadIdx.x; i < words; i += size_t(nblk) * blockDim.x)
      a.counts1[i] = 0u;
  }
  const uint32_t m = uint32_t(radix) - 1u;
  // four consecutive points a thread (a tile is kSortTile = 4 x 1024 points),
  // read as three 16-byte loads where the array is aligned, all issued before
  // the first shared-memory atomic
  static_assert(kSortTile == 4 * 1024, "1024 threads take four points each");
  const bool vec = (reinterpret_cast<uintptr_t>(a.xyz) & 15u) == 0;
  bool bad = false;
  for (int t = bid; t < tiles; t += nblk) {
    for (int d = threadIdx.x; d < radix; d += blockDim.x) ht[d] = 0;
    __syncthreads();
    const int p0 = t * kSortTile + 4 * int(threadIdx.x);
    int c[12];
    if (vec && p0 + 4 <= a.n) {
      const int4* q = reinterpret_cast<const int4*>(a.xyz + 3 * size_t(p0));
      const int4 v0 = q[0], v1 = q[1], v2 = q[2];
      c[0] = v0.x; c[1] = v0.y; c[2] = v0.z; c[3] = v0.w;
      c[4] = v1.x; c[5] = v1.y; c[6] = v1.z; c[7] = v1.w;
      c[8] = v2.x; c[9] = v2.y; c[10] = v2.z; c[11] = v2.w;
    } else {
#pragma unroll
      for (int j = 0; j < 12; ++j) c[j] = p0 + j / 3 < a.n ? a.xyz[3 * size_t(p0) + j] : 0;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (p0 + i >= a.n) break;
      const uint32_t xi = uint32_t(c[3 * i]), yi = uint32_t(c[3 * i + 1]), zi = uint32_t(c[3 * i + 2]);
      bad |= (xi > m) | (yi > m) | (zi > m);
      atomicAdd(&h[0][xi & m], 1u);
      atomicAdd(&h[1][yi & m], 1u);
      atomicAdd(&h[2][zi & m], 1u);
      atomicAdd(&ht[yi & m], 1u);
    }
    __syncthreads();
    if (a.counts0)
      for (int d = threadIdx.x; d < radix; d += blockDim.x) a.counts0[size_t(d) * tiles + t] = ht[d];
  }
  if (bad) atomicOr(&a.sc->status, kFlagRange);
  __syncthreads();
  for (int c = 0; c < 3; ++c)
    for (int d = threadIdx.x; d < radix; d += blockDim.x)
      if (h[c][d]) atomicAdd(&a.sc->chist[c][d], h[c][d]);
}

__global__ void __launch_bounds__(1024, 2) k_coord_hist(HistArgs a) {
  pdl_wait();
  coord_hist_body(a, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(1024, 2) k_coord_hist_seg(const __grid_constant__ Seg<HistArgs> s) {
  pdl_wait();
  const int f = seg_frame(s, blockIdx.x);
  coord_hist_body(s.a[f], blockIdx.x - s.start[f], s.start[f + 1] - s.start[f]);
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
__device__ __forceinline__ void tile_counts_body(const SortPassArgs& a, int t) {
  __shared__ uint32_t s_h[kMaxRadix];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int radix = 1 << a.bits;
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

__global__ void __launch_bounds__(kSortThreads) k_tile_counts(SortPassArgs a) {
  pdl_wait();
  tile_counts_body(a, blockIdx.x);
}

__global__ void __launch_bounds__(kSortThreads) k_tile_counts_seg(const __grid_constant__ Seg<SortPassArgs> s) {
  pdl_wait();
  const int f = seg_frame(s, blockIdx.x);
  tile_counts_body(s.a[f], blockIdx.x - s.start[f]);
}

// Scan: one warp per digit row.  counts become offsets: the start of the
// digit's bucket (total of the smaller digits) plus the counts of the earlier
// tiles.  Each lane owns a run of up to 8 consecutive tiles per batch.
__device__ __forceinline__ void tile_scan_body(const SortPassArgs& a, int bid) {
  const int lane = threadIdx.x & 31;
  const int radix = 1 << a.bits;
  const int d = bid * 8 + (threadIdx.x >> 5);
  if (d >= radix) return;
  uint32_t* r = a.counts + size_t(d) * a.tiles;
  constexpr int kRun = 8;
  // the first run of tile counts, loaded before the histogram so that the two
  // sets of loads are in flight together
  uint32_t c[kRun];
#pragma unroll
  for (int i = 0; i < kRun; ++i) {
    const int t = lane * kRun + i;
    c[i] = t < a.tiles ? r[t] : 0u;
  }
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
  for (int t0 = 0; t0 < a.tiles; t0 += 32 * kRun) {
    if (t0 > 0) {
#pragma unroll
      for (int i = 0; i < kRun; ++i) {
        const int t = t0 + lane * kRun + i;
        c[i] = t < a.tiles ? r[t] : 0u;
      }
    }
    uint32_t own = 0;
#pragma unroll
    for (int i = 0; i < kRun; ++i) own += c[i];
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

__global__ void __launch_bounds__(256) k_tile_scan(SortPassArgs a) {
  pdl_wait();
  tile_scan_body(a, blockIdx.x);
}

__global__ void __launch_bounds__(256) k_tile_scan_seg(const __grid_constant__ Seg<SortPassArgs> s) {
  pdl_wait();
  const int f = seg_frame(s, blockIdx.x);
  tile_scan_body(s.a[f], blockIdx.x - s.start[f]);
}

// Scatter: rank each key of the tile among equal digits (stable), then write
// the tile out in digit runs at the offsets the scan produced.
template <int THREADS>
__device__ __forceinline__ void sort_scatter_body(const SortPassArgs& a, int t) {
  using SS = ScatterShape<THREADS>;
  constexpr int kScatterWarps = SS::kWarps, kScatterKpt = SS::kKpt, kPairWords = SS::kPairWords;
  constexpr int kDigitsPerThread = SS::kDigitsPerThread;
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
  const int shift = a.shift;
  const int warp_base = t * kSortTile + warp * (32 * kScatterKpt);
  for (int i = tid; i < kPairWords * radix; i += THREADS) s_whist[i] = 0;
  // this tile's global start of every digit, known before any key is ranked
  for (int d = tid; d < radix; d += THREADS) s_gbase[d] = a.counts[size_t(d) * a.tiles + t];

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
    if (tid == THREADS - 1) *s_count = start;
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
      if (a.pos_out) {
        const uint32_t g = s_gbase[dj] + (lp - s_tstart[dj]);
        if (g < uint32_t(a.n)) a.pos_out[warp_base + j * 32 + lane] = int32_t(g);
      }
    }
  }
  __syncthreads();
  const uint32_t cnt = *s_count;
  uint32_t* ko = a.keys_out;
  uint32_t* vo = a.vals_out;
  int32_t* ro = a.rank_out;
  for (uint32_t i = tid; i < cnt; i += THREADS) {
    const uint32_t k = s_keys[i], v = s_vals[i];
    const uint32_t dk = (k >> shift) & m;
    const uint32_t g = s_gbase[dk] + (i - s_tstart[dk]);
    if (g >= uint32_t(a.n) || v >= uint32_t(a.n)) continue;
    if (ko) ko[g] = k;
    if (vo) vo[g] = v;
    if (ro) ro[v] = int32_t(g);
  }
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, ScatterShape<THREADS>::kMinBlocks) k_sort_scatter(SortPassArgs a) {
  pdl_wait();
  sort_scatter_body<THREADS>(a, blockIdx.x);
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, ScatterShape<THREADS>::kMinBlocks)
    k_sort_scatter_seg(const __grid_constant__ Seg<SortPassArgs> s) {
  pdl_wait();
  const int f = seg_frame(s, blockIdx.x);
  sort_scatter_body<THREADS>(s.a[f], blockIdx.x - s.start[f]);
}

// ---------------------------------------------------------------- slab sort
// One block per y-slab of the y-sorted (code, input index) pairs: sort the
// slab by (x, z) with two stable passes (z, then x), which gives the C3
// order.  A slab of up to kSlabMax points is held in shared memory and
// ranked kSlabKpt rounds per warp; warp w owns the contiguous positions
// [w C, (w + 1) C), so warp order is position order and the ballot ranks
// inside a warp keep lane order.  A larger slab (a cloud with very many points
// in one plane) takes the same ranking through global memory, kSlabThreads
// points at a time, with running digit offsets carried from chunk to chunk.
constexpr int kSlabThreads = 256;
constexpr int kSlabWarps = kSlabThreads / 32;
constexpr int kSlabKpt = 8;
constexpr int kSlabMax = kSlabThreads * kSlabKpt;  // 4096 points
constexpr int kSlabPairWords = kSlabWarps / 2;    // digit counter words (two warps each)
constexpr int kSlabDigits = kMaxRadix / kSlabThreads;  // digits owned by each thread

size_t slab_smem_bytes() {
  return sizeof(uint32_t) * (size_t(kSlabPairWords) * kMaxRadix + 2 * size_t(kSlabMax) + kMaxRadix + kSlabWarps + 4);
}

// exclusive scan of one value per thread over the 1024-thread block
__device__ __forceinline__ uint32_t slab_block_scan(uint32_t v, uint32_t* s_warp, uint32_t* total) {
  static_assert(kSlabWarps <= 32, "one warp scans the warp totals");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < kSlabWarps ? s_warp[lane] : 0u;
    uint32_t wx = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wx, o);
      if (lane >= o) wx += y;
    }
    if (lane < kSlabWarps) s_warp[lane] = wx - w;
    if (lane == 31 && total) *total = wx;
  }
  __syncthreads();
  const uint32_t r = s_warp[warp] + x - v;
  __syncthreads();
  return r;
}

// Stable rank of one key among the equal digits of its warp (lanes in order),
// added to the warp's digit counter (16-bit half `half` of the pair word).
__device__ __forceinline__ uint32_t warp_rank(bool valid, uint32_t d, int bits, uint32_t* wh, int half, int lane) {
  uint32_t peers = __ballot_sync(0xffffffffu, valid);
  for (int b = 0; b < bits; ++b) {
    const bool bit = (d >> b) & 1u;
    const uint32_t on = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? on : ~on;
  }
  const int leader = peers ? __ffs(peers) - 1 : lane;
  uint32_t old = 0;
  if (valid && lane == leader) old = (atomicAdd(&wh[d], uint32_t(__popc(peers)) << half) >> half) & 0xffffu;
  return __shfl_sync(0xffffffffu, old, leader) + __popc(peers & ((1u << lane) - 1u));
}

// For digit d (one per thread): the counters of the warps become their
// exclusive offsets; returns the digit's total.
__device__ __forceinline__ uint32_t digit_warp_offsets(uint32_t* cnt, int radix, int d) {
  uint32_t run = 0;
  if (d < radix) {
#pragma unroll
    for (int w = 0; w < kSlabPairWords; ++w) {
      const uint32_t c = cnt[w * radix + d];
      const uint32_t lo = c & 0xffffu, hi = c >> 16;
      cnt[w * radix + d] = run | ((run + lo) << 16);
      run += lo + hi;
    }
  }
  return run;
}

__device__ __forceinline__ void slab_sort_body(const SlabArgs& sa, int yv) {
  const int n = sa.n, bits = sa.bits;
  const uint32_t* __restrict__ keys_in = sa.keys_in;
  const uint32_t* __restrict__ vals_in = sa.vals_in;
  uint32_t* __restrict__ keys_tmp = sa.keys_tmp;
  uint32_t* __restrict__ vals_tmp = sa.vals_tmp;
  uint32_t* __restrict__ keys_out = sa.keys_out;
  int32_t* __restrict__ vals_out = sa.vals_out;
  const DevScalars* __restrict__ sc = sa.sc;
  extern __shared__ uint32_t smem[];
  uint32_t* cnt = smem;                                   // [kSlabPairWords][radix]
  uint32_t* s_keys = cnt + kSlabPairWords * kMaxRadix;    // [kSlabMax]
  uint32_t* s_vals = s_keys + kSlabMax;                   // [kSlabMax]
  uint32_t* s_start = s_vals + kSlabMax;                  // [radix]
  uint32_t* s_warp = s_start + kMaxRadix;                 // [kSlabWarps]
  uint32_t* s_misc = s_warp + kSlabWarps;                 // [4]

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int radix = 1 << bits;
  const uint32_t m = uint32_t(radix) - 1u;
  if (yv >= radix) return;
  const uint32_t* hy = sc->chist[1];
  const uint32_t size = hy[yv];
  if (size == 0) return;
  // the slab starts after every point of a smaller y
  uint32_t below = 0;
  for (int e = tid; e < yv; e += kSlabThreads) below += hy[e];
  slab_block_scan(below, s_warp, &s_misc[0]);
  const uint32_t start = s_misc[0];
  if (uint64_t(start) + size > uint64_t(n)) return;  // inconsistent histogram: leave the slab alone
  uint32_t* wh = cnt + (warp >> 1) * radix;
  const int half = 16 * (warp & 1);

  if (size <= uint32_t(kSlabMax)) {
    // the slab's z and x extents: each pass ranks the coordinate minus its
    // smallest value in the slab, with as many digit bits as the extent needs
    // (the order is the same; the digit counters and ballots are fewer)
    __shared__ uint32_t s_ext[4][kSlabWarps];
    uint32_t zlo = m, zhi = 0, xlo = m, xhi = 0;
    for (uint32_t i = tid; i < size; i += kSlabThreads) {
      const uint32_t key = keys_in[start + i];
      s_keys[i] = key;
      s_vals[i] = vals_in[start + i];
      const uint32_t z = (key >> (2 * bits)) & m, x = key & m;
      zlo = min(zlo, z);
      zhi = max(zhi, z);
      xlo = min(xlo, x);
      xhi = max(xhi, x);
    }
    zlo = __reduce_min_sync(0xffffffffu, zlo);
    zhi = __reduce_max_sync(0xffffffffu, zhi);
    xlo = __reduce_min_sync(0xffffffffu, xlo);
    xhi = __reduce_max_sync(0xffffffffu, xhi);
    if (lane == 0) {
      s_ext[0][warp] = zlo;
      s_ext[1][warp] = zhi;
      s_ext[2][warp] = xlo;
      s_ext[3][warp] = xhi;
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < kSlabWarps; ++w) {
      zlo = min(zlo, s_ext[0][w]);
      zhi = max(zhi, s_ext[1][w]);
      xlo = min(xlo, s_ext[2][w]);
      xhi = max(xhi, s_ext[3][w]);
    }
    const int chunk = int((size + 32 * kSlabWarps - 1) / (32 * kSlabWarps)) * 32;  // positions per warp
    const int rounds = chunk / 32;                                                 // <= kSlabKpt
    for (int pass = 0; pass < 2; ++pass) {
      const int shift = pass == 0 ? 2 * bits : 0;  // z, then x
      const uint32_t lo = pass == 0 ? zlo : xlo, ext = (pass == 0 ? zhi : xhi) - lo;
      const int dbits = max(1, 32 - __clz(int(ext)));  // digit bits of this pass (<= bits)
      const int pradix = 1 << dbits;
      uint32_t* pw = cnt + (warp >> 1) * pradix;       // this warp pair's counters
      for (int i = tid; i < kSlabPairWords * pradix; i += kSlabThreads) cnt[i] = 0;
      __syncthreads();
      uint32_t k[kSlabKpt], v[kSlabKpt], rk[kSlabKpt];
#pragma unroll
      for (int j = 0; j < kSlabKpt; ++j) {
        k[j] = v[j] = rk[j] = 0;
        if (j < rounds) {
          const uint32_t pos = uint32_t(warp * chunk + j * 32 + lane);
          const bool valid = pos < size;
          if (valid) {
            k[j] = s_keys[pos];
            v[j] = s_vals[pos];
          }
          rk[j] = warp_rank(valid, ((k[j] >> shift) & m) - lo, dbits, pw, half, lane);
          __syncwarp();
        }
      }
      __syncthreads();
      // each thread owns kSlabDigits consecutive digits
      uint32_t tot[kSlabDigits], own = 0;
#pragma unroll
      for (int i = 0; i < kSlabDigits; ++i) {
        tot[i] = digit_warp_offsets(cnt, pradix, kSlabDigits * tid + i);
        own += tot[i];
      }
      uint32_t ts = slab_block_scan(own, s_warp, nullptr);
#pragma unroll
      for (int i = 0; i < kSlabDigits; ++i) {
        if (kSlabDigits * tid + i < pradix) s_start[kSlabDigits * tid + i] = ts;
        ts += tot[i];
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kSlabKpt; ++j) {
        if (j < rounds) {
          const uint32_t pos = uint32_t(warp * chunk + j * 32 + lane);
          if (pos < size) {
            const uint32_t d = ((k[j] >> shift) & m) - lo;
            const uint32_t lp = s_start[d] + ((pw[d] >> half) & 0xffffu) + rk[j];
            if (lp < size) {
              s_keys[lp] = k[j];
              s_vals[lp] = v[j];
            }
          }
        }
      }
      __syncthreads();
    }
    for (uint32_t i = tid; i < size; i += kSlabThreads) {
      keys_out[start + i] = s_keys[i];
      vals_out[start + i] = int32_t(s_vals[i]);
    }
    if (sa.counts1) {
      // sort pass 1's tile counts (z digits of the C3 order): the slab's at
      // most kSlabMax positions lie in the 4096-key tiles t0 and t0 + 1, counted
      // in the digit counters (free after the last pass), then added to the totals
      const uint32_t t0 = start / kSortTile;
      const int tiles = (n + kSortTile - 1) / kSortTile;
      static_assert(kSlabMax <= kSortTile && 2 * kMaxRadix <= kSlabPairWords * kMaxRadix,
                    "a slab spans at most two tiles, counted in the digit counter words");
      // (z digits zlo .. zhi only)
      const int zr = int(zhi - zlo) + 1;
      for (int i = tid; i < 2 * zr; i += kSlabThreads) cnt[i] = 0;
      __syncthreads();
      for (uint32_t i = tid; i < size; i += kSlabThreads)
        atomicAdd(&cnt[((start + i) / kSortTile - t0) * zr + (((s_keys[i] >> (2 * bits)) & m) - zlo)], 1u);
      __syncthreads();
      for (int i = tid; i < 2 * zr; i += kSlabThreads) {
        const uint32_t c = cnt[i], t = t0 + uint32_t(i / zr);
        if (c && t < uint32_t(tiles)) atomicAdd(&sa.counts1[size_t(zlo + uint32_t(i % zr)) * tiles + t], c);
      }
    }
    return;
  }

  // ---- a slab larger than shared memory: the same passes, 1024 points at a
  // time, through global memory (pass 0 into the scratch arrays, pass 1 into
  // the final arrays)
  for (int pass = 0; pass < 2; ++pass) {
    const int shift = pass == 0 ? 2 * bits : 0;  // z, then x
    const uint32_t* ks = pass == 0 ? keys_in : keys_tmp;
    const uint32_t* vs = pass == 0 ? vals_in : vals_tmp;
    // digit histogram of the slab, then each digit's first position
    for (int d = tid; d < radix; d += kSlabThreads) s_start[d] = 0;
    __syncthreads();
    for (uint32_t i = tid; i < size; i += kSlabThreads) atomicAdd(&s_start[(ks[start + i] >> shift) & m], 1u);
    __syncthreads();
    // thread t: the next free positions of its kSlabDigits digits
    uint32_t run[kSlabDigits], own = 0;
#pragma unroll
    for (int i = 0; i < kSlabDigits; ++i) {
      run[i] = kSlabDigits * tid + i < radix ? s_start[kSlabDigits * tid + i] : 0u;
      own += run[i];
    }
    {
      uint32_t r0 = slab_block_scan(own, s_warp, nullptr);
#pragma unroll
      for (int i = 0; i < kSlabDigits; ++i) {
        const uint32_t h = run[i];
        run[i] = r0;
        r0 += h;
      }
    }
    for (uint32_t c0 = 0; c0 < size; c0 += kSlabThreads) {
      for (int i = tid; i < kSlabPairWords * radix; i += kSlabThreads) cnt[i] = 0;
#pragma unroll
      for (int i = 0; i < kSlabDigits; ++i)
        if (kSlabDigits * tid + i < radix) s_start[kSlabDigits * tid + i] = run[i];
      __syncthreads();
      const uint32_t pos = c0 + uint32_t(tid);
      const bool valid = pos < size;
      const uint32_t key = valid ? ks[start + pos] : 0u, val = valid ? vs[start + pos] : 0u;
      const uint32_t d = (key >> shift) & m;
      const uint32_t rk = warp_rank(valid, d, bits, wh, half, lane);
      __syncthreads();
      uint32_t tot[kSlabDigits];
#pragma unroll
      for (int i = 0; i < kSlabDigits; ++i) tot[i] = digit_warp_offsets(cnt, radix, kSlabDigits * tid + i);
      __syncthreads();
      if (valid) {
        const uint32_t lp = s_start[d] + ((wh[d] >> half) & 0xffffu) + rk;
        if (lp < size) {
          const uint32_t g = start + lp;
          if (pass == 0) {
            keys_tmp[g] = key;
            vals_tmp[g] = val;
          } else {
            keys_out[g] = key;
            vals_out[g] = int32_t(val);
            if (sa.counts1)  // sort pass 1's tile counts, one key at a time here
              atomicAdd(&sa.counts1[size_t((key >> (2 * bits)) & m) * ((n + kSortTile - 1) / kSortTile) +
                                    g / kSortTile],
                        1u);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < kSlabDigits; ++i) run[i] += tot[i];
      __syncthreads();
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSlabThreads, 4) k_slab_sort(SlabArgs a) {
  pdl_wait();
  slab_sort_body(a, blockIdx.x);
}

__global__ void __launch_bounds__(kSlabThreads, 4) k_slab_sort_seg(const __grid_constant__ Seg<SlabArgs> s) {
  pdl_wait();
  const int f = seg_frame(s, blockIdx.x);
  slab_sort_body(s.a[f], blockIdx.x - s.start[f]);
}

// One code's order per group of gx blocks (block x of code c).  Code 0 is the C1 order
// itself; codes 1 and 2 read the sorted ids along C2 and C3 and the packed C1
// codes in the same order (keys of the C2 pass; keys of the slab sort for C3),
// so only the C2 rank of a C3 point is a gather.  Each lane takes four
// consecutive positions (16-byte loads, the C2 rank gathers issued together);
// the neighbours across lanes come from shuffles, with one extra lookup at
// each end of the warp.
struct LinkPt {
  int k;       // sorted (C1) id, -1 outside [0, n)
  int r2;      // position in the C2 order (code 2 only)
  uint32_t c;  // packed C1 code
};

__device__ __forceinline__ LinkPt link_point(int r, int n, int code, const int32_t* __restrict__ ord,
                                             const uint32_t* keys, const int32_t* __restrict__ rank2) {
  LinkPt q{-1, -1, 0u};
  if (r < 0 || r >= n) return q;
  const int k = code == 0 ? r : ord[r];
  if (!in_range(k, n)) return q;
  q.k = k;
  q.c = keys[r];
  if (code == 2) q.r2 = rank2[k];
  return q;
}

__device__ __forceinline__ LinkPt shfl_pt(LinkPt p, int delta, bool up) {
  LinkPt q;
  q.k = up ? __shfl_up_sync(0xffffffffu, p.k, delta) : __shfl_down_sync(0xffffffffu, p.k, delta);
  q.r2 = up ? __shfl_up_sync(0xffffffffu, p.r2, delta) : __shfl_down_sync(0xffffffffu, p.r2, delta);
  q.c = up ? __shfl_up_sync(0xffffffffu, p.c, delta) : __shfl_down_sync(0xffffffffu, p.c, delta);
  return q;
}

constexpr int kLinkThreads = 256;
constexpr int kLinkPerLane = 4;

// whether two points lie on one scan line of `code` (equal in its two major coordinates)
__device__ __forceinline__ bool same_scan_line(int code, uint32_t a, uint32_t c, int b) {
  int ax, ay, az, cx, cy, cz;
  decode_c1(a, b, ax, ay, az);
  decode_c1(c, b, cx, cy, cz);
  if (code == 0) return az == cz && ay == cy;
  if (code == 1) return ax == cx && az == cz;
  return ay == cy && ax == cx;
}

// Under the same-line variant (same_line) a pair is linked along a code only on
// one scan line of it (k_c1_line_flags then records the missing C1 links).
template <bool SAME_LINE>
__device__ __forceinline__ void link_body(const LinkArgs& la, int bx, int gx, int code) {
  const int n = la.n, bits = la.bits, cap = la.cap;
  const int32_t* __restrict__ ord23 = la.ord23;
  const uint32_t* __restrict__ keys_c2 = la.keys_c2;
  const uint32_t* __restrict__ keys_c3 = la.keys_c3;
  const int32_t* __restrict__ rank2 = la.rank2;
  const uint32_t* __restrict__ pk = la.pk;
  int4* __restrict__ c4 = la.c4;
  DevScalars* __restrict__ sc = la.sc;
  __shared__ unsigned long long s_red[8];
  const int lane = threadIdx.x & 31;
  const int32_t* ord = code == 0 ? nullptr : ord23 + size_t(code - 1) * size_t(cap);
  const uint32_t* keys = code == 0 ? pk : (code == 1 ? keys_c2 : keys_c3);
  const bool vec = ((reinterpret_cast<uintptr_t>(ord) | reinterpret_cast<uintptr_t>(keys)) & 15u) == 0;
  unsigned long long edges = 0;
  float dist_f = 0.f;  // this thread's few edge lengths; converted to fixed point once
  constexpr int kSpan = 32 * kLinkPerLane;
  const int warps = gx * (kLinkThreads / 32);
  // whole warps step together so the shuffles see every lane
  for (int base = (bx * (kLinkThreads / 32) + (threadIdx.x >> 5)) * kSpan; base < n; base += warps * kSpan) {
    const int r0 = base + kLinkPerLane * lane;
    int kk[kLinkPerLane];
    uint32_t cc[kLinkPerLane];
    if (vec && r0 + kLinkPerLane <= n) {
      const uint4 kv = *reinterpret_cast<const uint4*>(keys + r0);
      cc[0] = kv.x;
      cc[1] = kv.y;
      cc[2] = kv.z;
      cc[3] = kv.w;
      if (code == 0) {
#pragma unroll
        for (int i = 0; i < kLinkPerLane; ++i) kk[i] = r0 + i;
      } else {
        const int4 ov = *reinterpret_cast<const int4*>(ord + r0);
        kk[0] = ov.x;
        kk[1] = ov.y;
        kk[2] = ov.z;
        kk[3] = ov.w;
      }
    } else {
#pragma unroll
      for (int i = 0; i < kLinkPerLane; ++i) {
        const int r = r0 + i;
        kk[i] = -1;
        cc[i] = 0u;
        if (r < n) {
          kk[i] = code == 0 ? r : ord[r];
          cc[i] = keys[r];
        }
      }
    }
    LinkPt p[kLinkPerLane];
#pragma unroll
    for (int i = 0; i < kLinkPerLane; ++i) {
      p[i].k = in_range(kk[i], n) ? kk[i] : -1;
      p[i].c = cc[i];
      p[i].r2 = (code == 2 && p[i].k >= 0) ? rank2[p[i].k] : -1;
    }
    LinkPt before = shfl_pt(p[kLinkPerLane - 1], 1, true);
    LinkPt after = shfl_pt(p[0], 1, false);
    if (lane == 0) before = link_point(r0 - 1, n, code, ord, keys, rank2);
    if (lane == 31) after = link_point(r0 + kLinkPerLane, n, code, ord, keys, rank2);
#pragma unroll
    for (int i = 0; i < kLinkPerLane; ++i) {
      const LinkPt me = p[i];
      const LinkPt prev = i == 0 ? before : p[i - 1];
      const LinkPt next = i == kLinkPerLane - 1 ? after : p[i + 1];
      if (me.k < 0) continue;
      constexpr bool sl = SAME_LINE;
      const bool next_ok = next.k >= 0 && (!sl || same_scan_line(code, me.c, next.c, bits));
      const bool prev_ok = prev.k >= 0 && (!sl || same_scan_line(code, me.c, prev.c, bits));
      // the edge to the next position: counted once, unless an earlier code links the pair
      // (C1: adjacent sorted ids; C2: adjacent C2 positions; each on one line under the variant)
      bool dup_next = true;
      if (next_ok) {
        dup_next = code > 0 && abs(me.k - next.k) == 1 && (!sl || same_scan_line(0, me.c, next.c, bits));
        if (code == 2) dup_next |= abs(me.r2 - next.r2) == 1 && (!sl || same_scan_line(1, me.c, next.c, bits));
        if (!dup_next) {
          edges += 1;
          dist_f += sqrtf(float(sq_dist_c1(me.c, next.c, bits)));
        }
      }
      if (code == 0) continue;
      bool dup_prev = true;
      if (prev_ok) {
        dup_prev = abs(me.k - prev.k) == 1 && (!sl || same_scan_line(0, me.c, prev.c, bits));
        if (code == 2) dup_prev |= abs(me.r2 - prev.r2) == 1 && (!sl || same_scan_line(1, me.c, prev.c, bits));
      }
      int2* slot = reinterpret_cast<int2*>(c4 + me.k) + (code - 1);
      *slot = make_int2(dup_prev ? -1 : prev.k, dup_next ? -1 : next.k);
    }
  }
  unsigned long long dist = (unsigned long long)__float2ull_rn(dist_f * float(1u << kDistShift));
  edges = block_sum_u64<kLinkThreads>(edges, s_red);
  dist = block_sum_u64<kLinkThreads>(dist, s_red);
  if (threadIdx.x == 0) {
    if (edges) atomicAdd(&sc->n_edges, edges);
    if (dist) atomicAdd(&sc->dist_fx, dist);
  }
}

template <bool SAME_LINE>
__global__ void __launch_bounds__(kLinkThreads, 6) k_link(LinkArgs a) {
  pdl_wait();
  link_body<SAME_LINE>(a, blockIdx.x, gridDim.x, blockIdx.y);
}

// segmented: frame f's blocks are three runs of equal length, one per code
template <bool SAME_LINE>
__global__ void __launch_bounds__(kLinkThreads, 6) k_link_seg(const __grid_constant__ Seg<LinkArgs> s) {
  pdl_wait();
  const int f = seg_frame(s, blockIdx.x);
  const int local = blockIdx.x - s.start[f], gx = (s.start[f + 1] - s.start[f]) / 3;
  link_body<SAME_LINE>(s.a[f], local % gx, gx, local / gx);
}

// Same-line variant: the missing links of every sorted point to its C1
// neighbours k - 1, k + 1 (not on its C1 scan line) go into the high bits of
// its packed code, where every kernel that takes k +- 1 as neighbours looks.
// (A neighbour's word may already carry its own bits when read: the
// coordinates are decoded through masks, so that does not matter.)
__device__ __forceinline__ void c1_line_flags_body(int n, int bits, uint32_t* pk, int bid, int nblk) {
  for (int k = bid * blockDim.x + threadIdx.x; k < n; k += nblk * blockDim.x) {
    const uint32_t c = pk[k] & kCoordMask;
    const bool prev_ok = k > 0 && same_scan_line(0, c, pk[k - 1], bits);
    const bool next_ok = k + 1 < n && same_scan_line(0, c, pk[k + 1], bits);
    pk[k] = c | (prev_ok ? 0u : kNoPrevLink) | (next_ok ? 0u : kNoNextLink);
  }
}

__global__ void __launch_bounds__(256) k_c1_line_flags(int n, int bits, uint32_t* pk) {
  pdl_wait();
  c1_line_flags_body(n, bits, pk, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) k_c1_line_flags_seg(const __grid_constant__ Seg<LinkArgs> s) {
  pdl_wait();
  const int f = seg_frame(s, blockIdx.x);
  c1_line_flags_body(s.a[f].n, s.a[f].bits, s.a[f].pk, blockIdx.x - s.start[f], s.start[f + 1] - s.start[f]);
}

// Windows w > 1 (Section 2.2 with w points linked on each side): one thread
// per (code l, position r) fills the slots of the point at r for code l, the
// points d = 1..w positions before and after it: C2/C3 d = 1 into c4, every
// code's d >= 2 into cx (C1 d = 1 stays implicit: k - 1, k + 1).  A pair that
// an earlier code links (C1: sorted ids at most w apart; C2: C2 positions at
// most w apart; each on one scan line under the same-line variant) is left
// out of the later code's slots, so the union graph is a set.  The decision
// is a function of the pair and the code, so both ends reach the same one.
// Each undirected edge is counted (and its length summed) once, from the
// earlier position.
__global__ void __launch_bounds__(256) k_link_wide(int n, int bits, int cap, int window, int same_line,
                                                  const int32_t* __restrict__ ord23,
                                                  const uint32_t* __restrict__ keys_c2,
                                                  const uint32_t* __restrict__ keys_c3,
                                                  const int32_t* __restrict__ rank2, const uint32_t* __restrict__ pk,
                                                  int4* __restrict__ c4, int32_t* __restrict__ cx, int cx_stride,
                                                  DevScalars* __restrict__ sc) {
  pdl_wait();
  __shared__ unsigned long long s_red[8];
  const int code = blockIdx.y;
  const int32_t* ord = code == 0 ? nullptr : ord23 + size_t(code - 1) * size_t(cap);
  const uint32_t* keys = code == 0 ? pk : (code == 1 ? keys_c2 : keys_c3);
  const bool sl = same_line != 0;
  unsigned long long edges = 0;
  float dist_f = 0.f;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    const int k = code == 0 ? r : ord[r];
    if (!in_range(k, n)) continue;
    const uint32_t c = keys[r] & kCoordMask;
    const int r2 = code == 2 ? rank2[k] : -1;
    for (int d = 1; d <= window; ++d) {
      int slot[2];
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        slot[side] = -1;
        const int rr = side ? r + d : r - d;
        if (rr < 0 || rr >= n) continue;
        const int o = code == 0 ? rr : ord[rr];
        if (!in_range(o, n)) continue;
        const uint32_t oc = keys[rr] & kCoordMask;
        if (sl && !same_scan_line(code, c, oc, bits)) continue;
        bool dup = false;
        if (code >= 1) dup = abs(k - o) <= window && (!sl || same_scan_line(0, c, oc, bits));
        if (code == 2 && !dup) {
          const int o2 = rank2[o];
          dup = abs(r2 - o2) <= window && (!sl || same_scan_line(1, c, oc, bits));
        }
        if (dup) continue;
        slot[side] = o;
        if (side) {
          edges += 1;
          dist_f += sqrtf(float(sq_dist_c1(c, oc, bits)));
        }
      }
      if (d == 1) {
        if (code > 0) reinterpret_cast<int2*>(c4 + k)[code - 1] = make_int2(slot[0], slot[1]);
      } else {
        const int s0 = 6 * (d - 2) + 2 * code;
        cx[size_t(s0) * size_t(cx_stride) + k] = slot[0];
        cx[size_t(s0 + 1) * size_t(cx_stride) + k] = slot[1];
      }
    }
  }
  unsigned long long dist = (unsigned long long)__float2ull_rn(dist_f * float(1u << kDistShift));
  edges = block_sum_u64<256>(edges, s_red);
  dist = block_sum_u64<256>(dist, s_red);
  if (threadIdx.x == 0) {
    if (edges) atomicAdd(&sc->n_edges, edges);
    if (dist) atomicAdd(&sc->dist_fx, dist);
  }
}

// Each sorted point's mean edge length (its neighbours from every slot), for
// the node and pair readings of sigma_g: written to node_sig (if set), and its
// fixed-point sum over the points that have edges, with their count, added to
// the build scalars.
__global__ void __launch_bounds__(256) k_node_sigma(int n, int bits, GraphBufs gb, DevScalars* __restrict__ sc) {
  pdl_wait();
  __shared__ unsigned long long s_red[8];
  unsigned long long sum = 0, cnt = 0;
  const int slots = 6 + gb.nx;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const uint32_t pkw = gb.pk[k];
    const int4 s4 = gb.c4[k];
    float len = 0.f;
    int deg = 0;
    for (int j = 0; j < slots; ++j) {
      const int o = neighbour_of(j, k, n, pkw, s4, gb.cx, gb.cx_stride);
      if (o < 0) continue;
      len += sqrtf(float(sq_dist_c1(pkw, gb.pk[o], bits)));
      deg += 1;
    }
    const float mean = deg ? len / float(deg) : 0.f;
    if (gb.node_sig) gb.node_sig[k] = mean;
    if (deg) {
      sum += __float2ull_rn(mean * float(1u << kDistShift));
      cnt += 1;
    }
  }
  sum = block_sum_u64<256>(sum, s_red);
  cnt = block_sum_u64<256>(cnt, s_red);
  if (threadIdx.x == 0) {
    if (sum) atomicAdd(&sc->node_fx, sum);
    if (cnt) atomicAdd(&sc->node_cnt, cnt);
  }
}

// The three orders in input indices: C1 from perm1, C2 and C3 through perm1.
__global__ void __launch_bounds__(256) k_orders_export(int n, int cap, const int32_t* __restrict__ perm1,
                                                       const int32_t* __restrict__ ord23, int32_t* __restrict__ out) {
  pdl_wait();
  const int stride = gridDim.x * blockDim.x;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    out[r] = perm1[r];
    const int k = ord23[r];
    out[size_t(n) + r] = in_range(k, n) ? perm1[k] : -1;
    const int k3 = ord23[size_t(cap) + r];
    out[2 * size_t(n) + r] = in_range(k3, n) ? perm1[k3] : -1;
  }
}

}  // namespace

namespace {
// blocks of one frame's launch of each kernel (the same in both paths)
// one 4096-point tile a block, up to two resident blocks per SM
int coord_hist_blocks(int n, int num_sms) {
  return n <= 0 ? 0 : std::max(1, std::min((n + kSortTile - 1) / kSortTile, 2 * num_sms));
}
int link_gx(int n, int num_sms) {
  // the three codes' blocks together fill the GPU once (6 resident blocks of 256 threads per SM)
  return std::max(1, std::min((n + kLinkThreads * kLinkPerLane - 1) / (kLinkThreads * kLinkPerLane), num_sms * 2));
}
int line_flag_blocks(int n, int num_sms) { return n <= 0 ? 0 : std::min((n + 255) / 256, num_sms * 8); }

template <int THREADS>
cudaError_t scatter_attr() {
  // the shared-memory limit is a per-device function attribute: set it once per device
  static std::atomic<unsigned long long> configured{0};
  return once_per_device(configured, [] {
    cudaError_t e = cudaFuncSetAttribute(k_sort_scatter<THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(scatter_smem_bytes(THREADS)));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_sort_scatter_seg<THREADS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               int(scatter_smem_bytes(THREADS)));
    return e;
  });
}

cudaError_t slab_attr() {
  static std::atomic<unsigned long long> configured{0};  // the shared-memory limit is set once per device
  return once_per_device(configured, [] {
    cudaError_t e = cudaFuncSetAttribute(k_slab_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, int(slab_smem_bytes()));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_slab_sort_seg, cudaFuncAttributeMaxDynamicSharedMemorySize, int(slab_smem_bytes()));
    return e;
  });
}

template <typename A, typename K>
cudaError_t launch_seg(K kernel, const A* args, const int* blocks, int count, int threads, size_t smem,
                       cudaStream_t stream) {
  if (count < 1 || count > kSegMax) return cudaErrorInvalidValue;
  Seg<A> sg;
  for (int f = 0; f < count; ++f) sg.a[f] = args[f];
  const int grid = seg_layout(sg, blocks, count);
  if (grid == 0) return cudaSuccess;
  return launch_kernel(kernel, dim3(grid), dim3(threads), smem, stream, false, sg);
}

SlabArgs slab_args(int n, int bits, int cap, const SortBufs& sb, const GraphBufs& gb, const DevScalars* sc) {
  // scratch for slabs larger than shared memory: the C2 order and C2 ranks, written later
  return SlabArgs{n,  bits, sb.keys[0], sb.vals[0], reinterpret_cast<uint32_t*>(gb.ord23),
                  reinterpret_cast<uint32_t*>(gb.rank2), sb.keys[1], gb.ord23 + size_t(cap), sc,
                  sb.tile_counts + sb.count_stride};
}
}  // namespace

HistArgs hist_args(const int32_t* xyz, int n, int bits, DevScalars* sc, const SortBufs& sb) {
  return HistArgs{xyz, n, bits, sc, sb.tile_counts, sb.tile_counts + sb.count_stride};
}

LinkArgs link_args(int n, int bits, int cap, const GraphBufs& gb, const SortBufs& sb, DevScalars* sc) {
  return LinkArgs{n, bits, cap, gb.ord23, sb.keys[0], sb.keys[1], gb.rank2, gb.pk, gb.c4, sc};
}

cudaError_t launch_coord_hist(const int32_t* xyz, int n, int bits, DevScalars* sc, const SortBufs* sb, int num_sms,
                              cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const HistArgs h = sb ? hist_args(xyz, n, bits, sc, *sb) : HistArgs{xyz, n, bits, sc, nullptr, nullptr};
  // one block a tile, two per SM: every tile of a 1M-point frame in one wave
  return launch_kernel(k_coord_hist, dim3(coord_hist_blocks(n, num_sms)), dim3(1024), 0, stream, false, h);
}

cudaError_t launch_tile_counts(const SortPassArgs& a, cudaStream_t stream) {
  return launch_kernel(k_tile_counts, dim3(a.tiles), dim3(kSortThreads), 0, stream, false, a);
}

cudaError_t launch_tile_scan(const SortPassArgs& a, cudaStream_t stream) {
  return launch_kernel(k_tile_scan, dim3(((1 << a.bits) + 7) / 8), dim3(256), 0, stream, false, a);
}

cudaError_t launch_sort_scatter(const SortPassArgs& a, cudaStream_t stream) {
  const cudaError_t e = scatter_attr<kScatterThreads>();
  if (e != cudaSuccess) return e;
  return launch_kernel(k_sort_scatter<kScatterThreads>, dim3(a.tiles), dim3(kScatterThreads),
                       scatter_smem_bytes(kScatterThreads), stream, false, a);
}

cudaError_t launch_sort_pass(const SortPassArgs& a, cudaStream_t stream) {
  cudaError_t e = pass_counted_before(a.pass) ? cudaSuccess : launch_tile_counts(a, stream);
  if (e == cudaSuccess) e = launch_tile_scan(a, stream);
  if (e == cudaSuccess) e = launch_sort_scatter(a, stream);
  return e;
}

cudaError_t launch_slab_sort(int n, int bits, int cap, const SortBufs& sb, const GraphBufs& gb,
                             const DevScalars* sc, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const cudaError_t e = slab_attr();
  if (e != cudaSuccess) return e;
  return launch_kernel(k_slab_sort, dim3(1 << bits), dim3(kSlabThreads), slab_smem_bytes(), stream, false,
                       slab_args(n, bits, cap, sb, gb, sc));
}

cudaError_t launch_link(int n, int bits, int cap, bool same_line, const GraphBufs& gb, const SortBufs& sb,
                        DevScalars* sc, int num_sms, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int gx = link_gx(n, num_sms);
  const LinkArgs la = link_args(n, bits, cap, gb, sb, sc);
  if (!same_line) return launch_kernel(k_link<false>, dim3(gx, 3), dim3(kLinkThreads), 0, stream, false, la);
  const cudaError_t e = launch_kernel(k_link<true>, dim3(gx, 3), dim3(kLinkThreads), 0, stream, false, la);
  if (e != cudaSuccess) return e;
  return launch_kernel(k_c1_line_flags, dim3(line_flag_blocks(n, num_sms)), dim3(256), 0, stream, false, n, bits,
                       gb.pk);
}

// ---- segmented (one launch over the frames of a batch)

cudaError_t launch_coord_hist_seg(const HistArgs* a, int count, int num_sms, cudaStream_t stream) {
  int blocks[kSegMax];
  for (int f = 0; f < count && f < kSegMax; ++f) blocks[f] = coord_hist_blocks(a[f].n, num_sms);
  return launch_seg(k_coord_hist_seg, a, blocks, count, 1024, 0, stream);
}

cudaError_t launch_sort_pass_seg(const SortPassArgs* a, int count, int scatter_threads, cudaStream_t stream) {
  int tiles[kSegMax], scan[kSegMax];
  for (int f = 0; f < count && f < kSegMax; ++f) {
    tiles[f] = a[f].n > 0 ? a[f].tiles : 0;
    scan[f] = a[f].n > 0 ? ((1 << a[f].bits) + 7) / 8 : 0;
  }
  cudaError_t e = count > 0 && pass_counted_before(a[0].pass)
                      ? cudaSuccess
                      : launch_seg(k_tile_counts_seg, a, tiles, count, kSortThreads, 0, stream);
  if (e == cudaSuccess) e = launch_seg(k_tile_scan_seg, a, scan, count, 256, 0, stream);
  if (e != cudaSuccess) return e;
  switch (scatter_threads) {
    case 256:
      e = scatter_attr<256>();
      return e != cudaSuccess ? e
                              : launch_seg(k_sort_scatter_seg<256>, a, tiles, count, 256, scatter_smem_bytes(256), stream);
    case 1024:
      e = scatter_attr<1024>();
      return e != cudaSuccess
                 ? e
                 : launch_seg(k_sort_scatter_seg<1024>, a, tiles, count, 1024, scatter_smem_bytes(1024), stream);
    default:
      e = scatter_attr<512>();
      return e != cudaSuccess ? e
                              : launch_seg(k_sort_scatter_seg<512>, a, tiles, count, 512, scatter_smem_bytes(512), stream);
  }
}

cudaError_t launch_slab_sort_seg(const int* n, const int* bits, const int* cap, const SortBufs* sb,
                                 const GraphBufs* gb, DevScalars* const* sc, int count, cudaStream_t stream) {
  if (count < 1 || count > kSegMax) return cudaErrorInvalidValue;
  const cudaError_t e = slab_attr();
  if (e != cudaSuccess) return e;
  SlabArgs a[kSegMax];
  int blocks[kSegMax];
  for (int f = 0; f < count; ++f) {
    a[f] = slab_args(n[f], bits[f], cap[f], sb[f], gb[f], sc[f]);
    blocks[f] = n[f] > 0 ? (1 << bits[f]) : 0;
  }
  return launch_seg(k_slab_sort_seg, a, blocks, count, kSlabThreads, slab_smem_bytes(), stream);
}

cudaError_t launch_link_seg(const LinkArgs* a, int count, bool same_line, int num_sms, cudaStream_t stream) {
  int blocks[kSegMax], flags[kSegMax];
  for (int f = 0; f < count && f < kSegMax; ++f) {
    blocks[f] = a[f].n > 0 ? 3 * link_gx(a[f].n, num_sms) : 0;
    flags[f] = line_flag_blocks(a[f].n, num_sms);
  }
  if (!same_line) return launch_seg(k_link_seg<false>, a, blocks, count, kLinkThreads, 0, stream);
  const cudaError_t e = launch_seg(k_link_seg<true>, a, blocks, count, kLinkThreads, 0, stream);
  if (e != cudaSuccess) return e;
  return launch_seg(k_c1_line_flags_seg, a, flags, count, 256, 0, stream);
}

cudaError_t launch_link_wide(int n, int bits, int cap, int window, bool same_line, const GraphBufs& gb,
                             const SortBufs& sb, DevScalars* sc, int num_sms, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  if (window < 2 || window > kMaxWindow || gb.nx != extra_slots(window) || !gb.cx) return cudaErrorInvalidValue;
  const int gx = std::max(1, std::min((n + 255) / 256, num_sms * 4));
  const cudaError_t e = launch_kernel(k_link_wide, dim3(gx, 3), dim3(256), 0, stream, false, n, bits, cap, window,
                                      same_line ? 1 : 0, gb.ord23, sb.keys[0], sb.keys[1], gb.rank2, gb.pk, gb.c4,
                                      gb.cx, gb.cx_stride, sc);
  if (e != cudaSuccess || !same_line) return e;
  return launch_kernel(k_c1_line_flags, dim3(std::min((n + 255) / 256, num_sms * 8)), dim3(256), 0, stream, false, n,
                       bits, gb.pk);
}

cudaError_t launch_node_sigma(int n, int bits, const GraphBufs& gb, DevScalars* sc, int num_sms, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = std::max(1, std::min((n + 255) / 256, num_sms * 8));
  return launch_kernel(k_node_sigma, dim3(grid), dim3(256), 0, stream, false, n, bits, gb, sc);
}

cudaError_t launch_orders_export(int n, int cap, const GraphBufs& gb, int32_t* out, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = std::max(1, std::min((n + 255) / 256, 152 * 16));
  return launch_kernel(k_orders_export, dim3(grid), dim3(256), 0, stream, false, n, cap, gb.perm1, gb.ord23, out);
}

SortPassArgs slg_pass_args(int pass, const int32_t* xyz, int n, int bits, int cap, const SortBufs& sb,
                           const GraphBufs& gb, const DevScalars* sc) {
  SortPassArgs a{};
  a.n = n;
  a.bits = bits;
  a.tiles = (n + kSortTile - 1) / kSortTile;
  a.pass = pass;
  a.counts = sb.tile_counts + size_t(pass) * sb.count_stride;
  a.sc = sc;
  if (pass == 0) {
    // y-slabs: keys are packed C1 codes, values input indices
    a.shift = bits;
    a.coord = 1;
    a.xyz = xyz;
    a.keys_out = sb.keys[0];
    a.vals_out = sb.vals[0];
    return a;
  }
  if (pass == 1) {
    // C1: the C3 order (from the slab sort) on z; ends with pk, perm1, rank1 and the C3
    // order as sorted ids
    a.shift = 2 * bits;
    a.coord = 2;
    a.keys_in = sb.keys[1];
    a.vals_in = reinterpret_cast<const uint32_t*>(gb.ord23 + size_t(cap));
    a.keys_out = gb.pk;
    a.vals_out = reinterpret_cast<uint32_t*>(gb.perm1);
    a.rank_out = gb.rank1;
    a.pos_out = gb.ord23 + size_t(cap);  // the C3 order now as sorted ids (over the input indices read here)
    return a;
  }
  // C2: the C1 order (value = position = sorted id) on x
  a.shift = 0;
  a.coord = 0;
  a.keys_in = gb.pk;
  a.vals_in = nullptr;
  a.keys_out = sb.keys[0];  // the packed codes along C2, for the link step
  a.vals_out = reinterpret_cast<uint32_t*>(gb.ord23);
  a.rank_out = gb.rank2;
  return a;
}

// ---------------------------------------------------------------- shared launch pieces

bool pdl_enabled() {
  static const bool on = std::getenv("FGBD_PDL") != nullptr;
  return on;
}

namespace {
__global__ void __launch_bounds__(256) k_zero_words(uint32_t* __restrict__ p, size_t words) {
  pdl_wait();
  for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < words; i += size_t(gridDim.x) * blockDim.x)
    p[i] = 0u;
}

__global__ void __launch_bounds__(256) k_zero_words_seg(const __grid_constant__ Seg<ZeroArgs> s) {
  pdl_wait();
  const int f = seg_frame(s, blockIdx.x);
  const size_t b = size_t(blockIdx.x - s.start[f]), nb = size_t(s.start[f + 1] - s.start[f]);
  for (size_t i = b * blockDim.x + threadIdx.x; i < s.a[f].words; i += nb * blockDim.x) s.a[f].p[i] = 0u;
}
}  // namespace

cudaError_t launch_zero_words_seg(const ZeroArgs* a, int count, cudaStream_t stream) {
  int blocks[kSegMax];
  for (int f = 0; f < count && f < kSegMax; ++f) blocks[f] = int(std::min<size_t>((a[f].words + 255) / 256, 64));
  return launch_seg(k_zero_words_seg, a, blocks, count, 256, 0, stream);
}

cudaError_t launch_zero_words(uint32_t* p, size_t words, cudaStream_t stream) {
  if (words == 0) return cudaSuccess;
  const int grid = int(std::min<size_t>((words + 255) / 256, 64));
  return launch_kernel(k_zero_words, dim3(grid), dim3(256), 0, stream, false, p, words);
}

}  // namespace fgbd
