// NE-GBP: noise estimation using graph-based patches (Section 2.3), plus the
// per-point colour spread that the limited region of FSLR uses (Section 2.4).
//
// k_gather_colors: colours of the caller (input order) into sorted order.
// k_ne_moments: per point, its patch {i} + neighbours.  The spread
//   (sigma_R + sigma_G + sigma_B)/3 is written for every point.  A point with
//   exactly 6 neighbours contributes the patch a_i = [f_i, f_n1, ..., f_n6],
//   neighbours in increasing distance (ties by offset (dz, dy, dx), then
//   index), to the first and second moments sum a and sum a a^T.  uint8
//   colours are centred on 128 (exact in float16), so the moments are exact
//   integer sums: mma.sync products with float32 partial sums, moved to int64
//   before they can lose a bit (gram_mma.cuh).
// k_ne_finalize: one block.  Sigma = S2/N - mu mu^T in float64; float32
//   eigenvector estimates from a Householder tridiagonalisation, Sturm
//   multisection and inverse iteration (tridiag.cuh); each eigenvalue is then
//   the float64 Rayleigh quotient v^T Sigma v / v^T v, whose error is second
//   order in the eigenvector error; the values are sorted descending and the
//   tail rule gives sigma_est.
#include <algorithm>
#include <atomic>

#include "eigen.cuh"
#include "gram_mma.cuh"
#include "select.cuh"
#include "tridiag.cuh"

namespace fgbd {
namespace {

constexpr int kTiles = 28;  // 3x3 output tiles covering the upper triangle of a 21x21 matrix

// Colours into sorted order: four consecutive sorted points per thread, their
// input indices read as one int4 and the twelve colour loads issued together.
__device__ __forceinline__ void perm_quad(const int32_t* __restrict__ perm1, int k0, int n, int (&pi)[4]) {
  if (k0 + 4 <= n) {
    const int4 v = *reinterpret_cast<const int4*>(perm1 + k0);
    pi[0] = v.x;
    pi[1] = v.y;
    pi[2] = v.z;
    pi[3] = v.w;
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) pi[i] = k0 + i < n ? perm1[k0 + i] : -1;
  }
}

__device__ __forceinline__ void gather_u8_body(const uint8_t* __restrict__ rgb, int n,
                                               const int32_t* __restrict__ perm1, uint32_t* __restrict__ y8,
                                               int bid, int nblk) {
  for (int k0 = 4 * (bid * blockDim.x + threadIdx.x); k0 < n; k0 += 4 * nblk * blockDim.x) {
    int pi[4];
    perm_quad(perm1, k0, n, pi);
    uint32_t c[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      c[i] = 0u;
      if (in_range(pi[i], n)) {
        const size_t b = 3 * size_t(pi[i]);
        c[i] = uint32_t(__ldg(rgb + b)) | (uint32_t(__ldg(rgb + b + 1)) << 8) | (uint32_t(__ldg(rgb + b + 2)) << 16);
      }
    }
    if (k0 + 4 <= n) {
      *reinterpret_cast<uint4*>(y8 + k0) = make_uint4(c[0], c[1], c[2], c[3]);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (k0 + i < n) y8[k0 + i] = c[i];
    }
  }
}

__device__ __forceinline__ void gather_f32_body(const float* __restrict__ rgb, int n,
                                                const int32_t* __restrict__ perm1, float4* __restrict__ yf, int bid,
                                                int nblk) {
  for (int k0 = 4 * (bid * blockDim.x + threadIdx.x); k0 < n; k0 += 4 * nblk * blockDim.x) {
    int pi[4];
    perm_quad(perm1, k0, n, pi);
    float4 c[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      c[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (in_range(pi[i], n)) {
        const size_t b = 3 * size_t(pi[i]);
        c[i] = make_float4(__ldg(rgb + b), __ldg(rgb + b + 1), __ldg(rgb + b + 2), 0.f);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (k0 + i < n) yf[k0 + i] = c[i];
  }
}

__global__ void __launch_bounds__(256) k_gather_u8(const uint8_t* __restrict__ rgb, int n,
                                                   const int32_t* __restrict__ perm1,
                                                   uint32_t* __restrict__ y8) {
  pdl_wait();
  gather_u8_body(rgb, n, perm1, y8, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) k_gather_f32(const float* __restrict__ rgb, int n,
                                                    const int32_t* __restrict__ perm1,
                                                    float4* __restrict__ yf) {
  pdl_wait();
  gather_f32_body(rgb, n, perm1, yf, blockIdx.x, gridDim.x);
}

__global__ void __launch_bounds__(256) k_gather_seg(const __grid_constant__ Seg<GatherArgs> s) {
  pdl_wait();
  const int f = seg_frame(s, blockIdx.x);
  const GatherArgs& a = s.a[f];
  const int bid = blockIdx.x - s.start[f], nblk = s.start[f + 1] - s.start[f];
  if (a.dtype == 0) gather_u8_body(static_cast<const uint8_t*>(a.rgb), a.n, a.perm1, a.y8, bid, nblk);
  else gather_f32_body(static_cast<const float*>(a.rgb), a.n, a.perm1, a.yf, bid, nblk);
}

__device__ __forceinline__ void tile_rc(int tile, int& r0, int& c0) {
  // tiles (ti, tj), ti <= tj, of a 7x7 grid of 3x3 blocks, row-major
  int ti = 0, rem = tile;
  while (rem >= 7 - ti) {
    rem -= 7 - ti;
    ++ti;
  }
  r0 = 3 * ti;
  c0 = 3 * (ti + rem);
}

// one neighbour of a patch: sort key (d^2, dz, dy, dx packed so that integer
// order is lexicographic), its sorted id (input order among repeated voxels)
// and its colour, carried through the sort
template <int DT>
struct NbKey;
template <>
struct NbKey<0> {
  unsigned long long key;
  int idx;
  uint32_t col;  // packed R, G, B bytes
};
template <>
struct NbKey<1> {
  unsigned long long key;
  int idx;
  float r, g, b;
};


constexpr int kNeWarps = kNeThreads / 32;
// uint8 colours: the batch's patches as float16, entry-major: rows 0..20 the
// entries, row 21 the constant 1 of each valid patch, rows 22..31 zero (the
// second 16-row block of the mma tiles); 32 patches and 8 halves of padding a
// row (80-byte rows: the eight rows of an ldmatrix tile fall in distinct banks)
constexpr int kHRow = 40;
constexpr int kHRows = 32;
constexpr int kRowFloats = 33;  // 32 float entries, padded likewise
constexpr int kFirstLanes = 32 - kTiles;  // lanes 28..31 sum the first moments

// Per point: FSLR spread over the point and its neighbours (written to
// spread[k]) and, for a point with exactly 6 neighbours, its patch (the point
// then its neighbours by (d^2, dz, dy, dx, index)) written to column `lane`
// of the warp's transposed patch block.  Returns whether a patch was written.
template <int DT>
__device__ __forceinline__ bool point_patch(int k, int n, int bits, int lane, const uint32_t* __restrict__ pk,
                                            const int4* __restrict__ c4, const uint32_t* __restrict__ y8,
                                            const float4* __restrict__ yf, float* __restrict__ spread,
                                            float4* __restrict__ x0, bool moments, bool sorted_patches, __half* ath,
                                            float* atf) {
  int nb[6];
  bool v[6];
  const uint32_t pkk = pk[k];  // packed code, with the same-line variant's missing-C1-link bits
  nb[0] = k - 1;
  v[0] = c1_prev_linked(pkk, k);
  nb[1] = k + 1;
  v[1] = c1_next_linked(pkk, k, n);
  const int4 s = c4[k];
  nb[2] = s.x;
  nb[3] = s.y;
  nb[4] = s.z;
  nb[5] = s.w;
  v[2] = in_range(s.x, n);
  v[3] = in_range(s.y, n);
  v[4] = in_range(s.z, n);
  v[5] = in_range(s.w, n);
  int deg = 0;
#pragma unroll
  for (int j = 0; j < 6; ++j) deg += v[j];
  const bool patch = moments && deg == 6;
  NbKey<DT> e[6];
  uint32_t cpk[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int q = v[j] ? nb[j] : k;
    cpk[j] = patch ? pk[q] : 0u;
    e[j].idx = q;
    if (DT == 0) {
      reinterpret_cast<NbKey<0>&>(e[j]).col = y8[q];
    } else {
      const float4 c = yf[q];
      reinterpret_cast<NbKey<1>&>(e[j]).r = c.x;
      reinterpret_cast<NbKey<1>&>(e[j]).g = c.y;
      reinterpret_cast<NbKey<1>&>(e[j]).b = c.z;
    }
  }
  float sp;
  const float cnt = float(deg + 1);
  uint32_t own8 = 0;
  float ownr = 0.f, owng = 0.f, ownb = 0.f;
  if (DT == 0) {
    own8 = y8[k];
    if (x0)
      x0[k] = make_float4(float(own8 & 255u), float((own8 >> 8) & 255u), float((own8 >> 16) & 255u),
                          __uint_as_float(pkk));
    int sr = int(own8 & 255u), sg = int((own8 >> 8) & 255u), sb = int((own8 >> 16) & 255u);
    int qr = sr * sr, qg = sg * sg, qb = sb * sb;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      if (v[j]) {
        const uint32_t c = reinterpret_cast<NbKey<0>&>(e[j]).col;
        const int a = int(c & 255u), b = int((c >> 8) & 255u), d = int((c >> 16) & 255u);
        sr += a;
        sg += b;
        sb += d;
        qr += a * a;
        qg += b * b;
        qb += d * d;
      }
    }
    // cnt^2 times each population variance is an exact integer; the mean of
    // the three standard deviations is (sum of their roots) / (3 cnt), with one
    // rounded reciprocal instead of four divisions (a few ulp in all, far
    // inside the band in which the selection decides exactly)
    const int nn = deg + 1;
    const float vr = float(nn * qr - sr * sr), vg = float(nn * qg - sg * sg), vb = float(nn * qb - sb * sb);
    sp = (sqrtf(vr) + sqrtf(vg) + sqrtf(vb)) * __frcp_rn(3.0f * cnt);
  } else {
    const float4 o = yf[k];
    ownr = o.x;
    owng = o.y;
    ownb = o.z;
    if (x0) x0[k] = make_float4(ownr, owng, ownb, __uint_as_float(pkk));
    float mr = ownr, mg = owng, mb = ownb;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      if (v[j]) {
        const NbKey<1>& f = reinterpret_cast<NbKey<1>&>(e[j]);
        mr += f.r;
        mg += f.g;
        mb += f.b;
      }
    }
    const float icnt = __frcp_rn(cnt);
    mr *= icnt;
    mg *= icnt;
    mb *= icnt;
    float vr = (ownr - mr) * (ownr - mr), vg = (owng - mg) * (owng - mg), vb = (ownb - mb) * (ownb - mb);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      if (v[j]) {
        const NbKey<1>& f = reinterpret_cast<NbKey<1>&>(e[j]);
        vr += (f.r - mr) * (f.r - mr);
        vg += (f.g - mg) * (f.g - mg);
        vb += (f.b - mb) * (f.b - mb);
      }
    }
    sp = (sqrtf(vr * icnt) + sqrtf(vg * icnt) + sqrtf(vb * icnt)) * (1.0f / 3.0f);
  }
  spread[k] = sp;
  if (!patch) return false;

  int kx, ky, kz;
  decode_c1(pkk, bits, kx, ky, kz);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    int x, y, z;
    decode_c1(cpk[j], bits, x, y, z);
    const int dx = x - kx, dy = y - ky, dz = z - kz;
    const unsigned long long d2 = (unsigned long long)(dx * dx + dy * dy + dz * dz);
    e[j].key = (d2 << 33) | ((unsigned long long)(dz + 1024) << 22) | ((unsigned long long)(dy + 1024) << 11) |
               (unsigned long long)(dx + 1024);
  }
  // the place of each neighbour in the patch: its rank in the strict order
  // (key, index), from the 15 pairwise comparisons, so the colours are written
  // straight to their rows (the unique sorted order).  Without sorting (the
  // "w/o sort" ablation) the entries stay in link order: C1 prev, C1 next,
  // C2 prev, C2 next, C3 prev, C3 next.
  int rk[6] = {0, 1, 2, 3, 4, 5};
  if (sorted_patches) {
#pragma unroll
    for (int j = 0; j < 6; ++j) rk[j] = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = i + 1; j < 6; ++j) {
        const bool j_first = (e[j].key < e[i].key) || (e[j].key == e[i].key && e[j].idx < e[i].idx);
        rk[i] += j_first;
        rk[j] += !j_first;
      }
  }
  if (DT == 0) {
    // entry r of the patch, centred on 128 (exact in float16)
    ath[0 * kHRow + lane] = __int2half_rn(int(own8 & 255u) - 128);
    ath[1 * kHRow + lane] = __int2half_rn(int((own8 >> 8) & 255u) - 128);
    ath[2 * kHRow + lane] = __int2half_rn(int((own8 >> 16) & 255u) - 128);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const uint32_t c = reinterpret_cast<NbKey<0>&>(e[j]).col;
      __half* row = ath + (3 + 3 * rk[j]) * kHRow + lane;
      row[0] = __int2half_rn(int(c & 255u) - 128);
      row[kHRow] = __int2half_rn(int((c >> 8) & 255u) - 128);
      row[2 * kHRow] = __int2half_rn(int((c >> 16) & 255u) - 128);
    }
  } else {
    atf[0 * kRowFloats + lane] = ownr - 128.f;
    atf[1 * kRowFloats + lane] = owng - 128.f;
    atf[2 * kRowFloats + lane] = ownb - 128.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const NbKey<1>& f = reinterpret_cast<NbKey<1>&>(e[j]);
      float* row = atf + (3 + 3 * rk[j]) * kRowFloats + lane;
      row[0] = f.r - 128.f;
      row[kRowFloats] = f.g - 128.f;
      row[2 * kRowFloats] = f.b - 128.f;
    }
  }
  return true;
}

// Warp-synchronous: each warp takes 32 points at a time, stages their patches
// transposed in its own shared-memory block and accumulates the moments with
// __syncwarp only.  uint8 colours: float16 patches and mma.sync on the tensor
// pipe (gram_mma.cuh): per 16 patches four m16n8k16 products cover the upper
// triangle of the 22 x 22 Gram matrix of (a, 1), moved to exact int64 sums
// every kGramFlushPatches patches.  Float colours: lanes 0..27 own one 3x3
// tile of the upper triangle of sum a a^T, lanes 28..31 rows of sum a, in
// fp32 over 4 batches, then float64.  The block combines its warps through
// shared atomics and adds its totals to the context (uint8) or writes them
// (float).
template <int DT>
__device__ __forceinline__ void ne_moments_body(const MomentArgs& ma, int bid, int nblk) {
  const int n = ma.n, bits = ma.bits, moments = ma.moments, sorted_patches = ma.sorted_patches;
  const uint32_t* __restrict__ pk = ma.pk;
  const int4* __restrict__ c4 = ma.c4;
  const uint32_t* __restrict__ y8 = ma.y8;
  const float4* __restrict__ yf = ma.yf;
  float* __restrict__ spread = ma.spread;
  double* __restrict__ f64_partials = ma.f64_partials;
  DevScalars* __restrict__ sc = ma.sc;
  constexpr int kP = kD * kD + kD + 1;
  static_assert(kD + 1 <= kHRows && kHRows == 32, "entries, the constant row and the zero rows fill two 16-row blocks");
  __shared__ __align__(16) __half s_h[DT == 0 ? kNeWarps : 1][kHRows * kHRow];
  __shared__ __align__(16) float s_atf[DT == 1 ? kNeWarps : 1][kD * kRowFloats];
  __shared__ unsigned long long s_tot8[DT == 0 ? kP : 1];
  __shared__ double s_totf[DT == 1 ? kP : 1];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (moments) {
    for (int i = threadIdx.x; i < kP; i += kNeThreads) {
      if (DT == 0) s_tot8[i] = 0ull;
      else s_totf[i] = 0.0;
    }
    if (DT == 0) {
      // the warp's staging block: all zero (rows 22..31 stay so)
      uint32_t* hw = reinterpret_cast<uint32_t*>(&s_h[warp][0]);
      for (int i = lane; i < kHRows * kHRow / 2; i += 32) hw[i] = 0u;
    }
  }
  // the graph's Eq. 4 exponent scale, once, for the filter steps that follow
  // (float64 work, here off their critical path)
  if (bid == 0 && threadIdx.x == 0 && !sc->cexp_ready) {
    sc->cexp = step_cexp(sc);
    __threadfence();
    sc->cexp_ready = 1u;
  }
  __syncthreads();
  int r0 = 0, c0 = 0, rb = 0, re = 0;
  if (DT == 1) {
    if (lane < kTiles) {
      tile_rc(lane, r0, c0);
    } else {
      rb = ((lane - kTiles) * kD) / kFirstLanes;
      re = ((lane - kTiles + 1) * kD) / kFirstLanes;
    }
  }
  float gc[4][4] = {};  // uint8: the Gram blocks (m0, n0), (m0, n1), (m0, n2), (m1, n2)
  float accf[9] = {};
  double accd[9] = {};
  unsigned long long npatch = 0;
  int since_flush = 0;
  __half* ath = &s_h[DT == 0 ? warp : 0][0];
  float* atf = &s_atf[DT == 1 ? warp : 0][0];
  const uint32_t hbase = uint32_t(__cvta_generic_to_shared(ath));

  const int nwarps = nblk * kNeWarps;
  for (int base = (bid * kNeWarps + warp) * 32; base < n; base += nwarps * 32) {
    const int k = base + lane;
    bool has = false;
    if (k < n)
      has = point_patch<DT>(k, n, bits, lane, pk, c4, y8, yf, spread, ma.x0, moments != 0, sorted_patches != 0, ath,
                            atf);
    if (!moments) continue;
    if (DT == 0) {
      if (!has) {
#pragma unroll
        for (int r = 0; r < kD; ++r) ath[r * kHRow + lane] = __float2half_rn(0.f);
      }
      ath[kD * kHRow + lane] = __float2half_rn(has ? 1.f : 0.f);
    } else if (!has) {
#pragma unroll
      for (int r = 0; r < kD; ++r) atf[r * kRowFloats + lane] = 0.f;
    }
    const uint32_t hb = __ballot_sync(0xffffffffu, has);
    npatch += __popc(hb);
    __syncwarp();
    if (DT == 0) {
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        uint32_t lo[4], hi[4];
        ldsm_x4(gram_tile_addr(hbase, 0, 16 * ks, kHRow, lane), lo);
        ldsm_x4(gram_tile_addr(hbase, 16, 16 * ks, kHRow, lane), hi);
        mma_16816(gc[0], lo, lo[0], lo[2]);
        mma_16816(gc[1], lo, lo[1], lo[3]);
        mma_16816(gc[2], lo, hi[0], hi[2]);
        mma_16816(gc[3], hi, hi[0], hi[2]);
      }
      if (++since_flush == kGramFlushPatches / 32) {
        gram_flush(gc[0], 0, 0, kD + 1, lane, s_tot8, s_tot8 + kD * kD);
        gram_flush(gc[1], 0, 1, kD + 1, lane, s_tot8, s_tot8 + kD * kD);
        gram_flush(gc[2], 0, 2, kD + 1, lane, s_tot8, s_tot8 + kD * kD);
        gram_flush(gc[3], 1, 2, kD + 1, lane, s_tot8, s_tot8 + kD * kD);
        since_flush = 0;
      }
    } else {
      if (lane < kTiles) {
#pragma unroll 4
        for (int p = 0; p < 32; ++p) {
          float a[3], b[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            a[i] = atf[(r0 + i) * kRowFloats + p];
            b[i] = atf[(c0 + i) * kRowFloats + p];
          }
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) accf[3 * i + j] = fmaf(a[i], b[j], accf[3 * i + j]);
        }
      } else {
#pragma unroll
        for (int t = 0; t < 6; ++t) {
          const int r = rb + t;
          if (r < re) {
            float sum = 0.f;
            for (int p = 0; p < 32; ++p) sum += atf[r * kRowFloats + p];
            accf[t] += sum;
          }
        }
      }
      if (++since_flush == 4) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          accd[i] += double(accf[i]);
          accf[i] = 0.f;
        }
        since_flush = 0;
      }
    }
    __syncwarp();
  }
  if (!moments) return;
  // combine the warps of the block
  if (DT == 0) {
    gram_flush(gc[0], 0, 0, kD + 1, lane, s_tot8, s_tot8 + kD * kD);
    gram_flush(gc[1], 0, 1, kD + 1, lane, s_tot8, s_tot8 + kD * kD);
    gram_flush(gc[2], 0, 2, kD + 1, lane, s_tot8, s_tot8 + kD * kD);
    gram_flush(gc[3], 1, 2, kD + 1, lane, s_tot8, s_tot8 + kD * kD);
  } else {
#pragma unroll
    for (int i = 0; i < 9; ++i) accd[i] += double(accf[i]);
    if (lane < kTiles) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) atomicAdd(&s_totf[(r0 + i) * kD + (c0 + j)], accd[3 * i + j]);
    } else {
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        const int r = rb + t;
        if (r < re) atomicAdd(&s_totf[kD * kD + r], accd[t]);
      }
    }
  }
  if (lane == 0) {
    if (DT == 0) atomicAdd(&s_tot8[kD * kD + kD], npatch);
    else atomicAdd(&s_totf[kD * kD + kD], double(npatch));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kP; i += kNeThreads) {
    if (DT == 0) {
      const unsigned long long v = s_tot8[i];
      if (v == 0) continue;
      if (i < kD * kD) atomicAdd(reinterpret_cast<unsigned long long*>(&sc->s2[i]), v);
      else if (i < kD * kD + kD) atomicAdd(reinterpret_cast<unsigned long long*>(&sc->s1[i - kD * kD]), v);
      else atomicAdd(&sc->n_patches, v);
    } else {
      f64_partials[size_t(bid) * kP + i] = s_totf[i];
    }
  }
}

template <int DT>
__global__ void __launch_bounds__(kNeThreads, 4) k_ne_moments(MomentArgs a) {
  pdl_wait();
  ne_moments_body<DT>(a, blockIdx.x, gridDim.x);
}

template <int DT>
__global__ void __launch_bounds__(kNeThreads, 4) k_ne_moments_seg(const __grid_constant__ Seg<MomentArgs> s) {
  pdl_wait();
  const int f = seg_frame(s, blockIdx.x);
  ne_moments_body<DT>(s.a[f], blockIdx.x - s.start[f], s.start[f + 1] - s.start[f]);
}

// ---------------------------------------------------------------- finalize

constexpr int kFinThreads = 384;      // 12 warps

// barriers of the first kFinThreads threads of a block (barrier 1; 0 is __syncthreads)
__device__ __forceinline__ void fin_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kFinThreads) : "memory"); }

struct FinBar {
  __device__ void operator()() const { fin_bar(); }
};

// The eigenvalues of the D x D covariance S (float64, row-major in shared
// memory; Sf its float32 copy) as float64 Rayleigh quotients of float32
// eigenvector estimates (tridiag.cuh), sorted descending, then the tail rule:
// sigma_est and the eigenvalues into the context's scalars.  Threads
// 0..kFinThreads-1 of the block.
template <int D>
__device__ void eig_tail(const double* __restrict__ S, const float* __restrict__ Sf, DevScalars* __restrict__ sc,
                         double* __restrict__ sigma_out, int dtype) {
  static_assert(D <= 32, "warp 0 holds one eigenvalue a lane");
  __shared__ float V[D * D];  // eigenvector estimates (columns)
  __shared__ float s_mu[D];   // their float32 eigenvalues (the fallback of a non-finite quotient)
  __shared__ TridiagSmem<D, kFinThreads> tw;
  __shared__ long long s_key[D];
  __shared__ double s_sorted[D];
  __shared__ double s_num[D][D];
  __shared__ double V64[D][D + 1];
  const int tid = threadIdx.x;

  // float32 eigenvector estimates: Householder tridiagonalisation, Sturm
  // multisection and inverse iteration (tridiag.cuh)
  eig_vectors_f32<D, kFinThreads>(Sf, tw, V, s_mu, FinBar{});

  // float64 Rayleigh quotients of the eigenvector estimates.  float64 has a
  // long latency here, so the sums run as three interleaved chains.
  for (int e = tid; e < D * D; e += kFinThreads) V64[e / D][e % D] = double(V[e]);
  fin_bar();
  for (int e = tid; e < D * D; e += kFinThreads) {
    const int k = e / D, r = e % D;
    double w0 = 0.0, w1 = 0.0, w2 = 0.0;
#pragma unroll
    for (int c = 0; c < D; c += 3) {
      w0 = fma(S[r * D + c], V64[c][k], w0);
      if (c + 1 < D) w1 = fma(S[r * D + c + 1], V64[c + 1][k], w1);
      if (c + 2 < D) w2 = fma(S[r * D + c + 2], V64[c + 2][k], w2);
    }
    s_num[k][r] = (w0 + w1 + w2) * V64[r][k];
  }
  fin_bar();
  // the rest runs in warp 0, lane j < D holding eigenvalue j
  if (tid < 32) {
    constexpr unsigned kFull = 0xffffffffu;
    const int lane = tid;
    double lam = 0.0;
    if (lane < D) {
      double n0 = 0.0, n1 = 0.0, n2 = 0.0, d0 = 0.0, d1 = 0.0, d2 = 0.0;
#pragma unroll
      for (int r = 0; r < D; r += 3) {
        n0 += s_num[lane][r];
        d0 = fma(V64[r][lane], V64[r][lane], d0);
        if (r + 1 < D) {
          n1 += s_num[lane][r + 1];
          d1 = fma(V64[r + 1][lane], V64[r + 1][lane], d1);
        }
        if (r + 2 < D) {
          n2 += s_num[lane][r + 2];
          d2 = fma(V64[r + 2][lane], V64[r + 2][lane], d2);
        }
      }
      lam = div_newton(n0 + n1 + n2, d0 + d1 + d2);
      if (!isfinite(lam)) lam = double(s_mu[lane]);
    }
    // eigenvalues below 1e-9 max(lambda_1, 1) are numerical zeros (a rank-deficient
    // covariance); they are set to exactly 0 so the tail rule never decides on rounding noise
    double top = lane < D ? lam : -1.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) top = fmax(top, __shfl_xor_sync(kFull, top, o));
    if (lane < D && fabs(lam) < kZeroEigRel * fmax(top, 1.0)) lam = 0.0;
    // descending order (ties by index), by counting the larger values
    // (float64 compares are slow here: the values are compared through
    // order-preserving 64-bit integer keys of their bit patterns)
    if (lane < D) s_key[lane] = order_key(lam);
    __syncwarp();
    if (lane < D) {
      const long long mine = order_key(lam);
      int rank = 0;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const long long o = s_key[j];
        rank += (o > mine) || (o == mine && j < lane);
      }
      s_sorted[rank] = lam;
    }
    __syncwarp();
    const double sorted = lane < D ? s_sorted[lane] : 0.0;
    if (lane < D) sc->eig[lane] = sorted;
    // tail sums lambda_j + ... + lambda_D by a suffix scan (a tail of exact
    // zeros sums to exactly 0 in any order)
    double suffix = sorted;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double t = __shfl_down_sync(kFull, suffix, o);
      if (lane + o < D) suffix += t;
    }
    // tail rule, every m tested at once: the smallest m with
    // mean(lambda_{m+1..D}) <= median(lambda_{m+1..D}), tested as
    // sum <= median * count; m = D - 1 always passes
    bool pass = false;
    if (lane < D) {
      const int cnt = D - lane;
      const double med = (cnt & 1) ? s_sorted[lane + cnt / 2]
                                   : 0.5 * (s_sorted[lane + cnt / 2 - 1] + s_sorted[lane + cnt / 2]);
      pass = suffix <= med * double(cnt);
    }
    const int m = __ffs(__ballot_sync(kFull, pass)) - 1;
    const double tail = __shfl_sync(kFull, suffix, m);
    if (lane == 0) {
      const double tau = div_newton(tail, double(D - m));
      const double sg = sqrt(fmax(tau, 0.0));
      sc->m = m;
      sc->tau = tau;
      sc->sigma_est = sg;
      sc->ne_valid = 1;
      // the selection's FSLR threshold of this sigma_est, formed here where it
      // is off the critical path (float64)
      fslr_band(sc->fslr_factor, sg, dtype, sc->fslr_thr);
      sc->fslr_ready = 1u;
      if (sigma_out) *sigma_out = sg;
      __threadfence();
      atomicExch(&sc->sigma_ready, 1u);
    }
  }
}

// sigma_est from the patch moments, by the first kFinThreads threads of one
// block (its barriers count those threads only, so the rest of a larger block
// may leave at once).  With sc->pooled_patch, the per-channel patches of
// D = 7 pooled over the channels (a reading of Section 2.3), built from the
// same sums: channel c's sums are the entries 3i + c of the RGB moments.
__device__ __noinline__ void finalize_block(int dtype, const double* __restrict__ f64_partials, int nblocks,
                                            DevScalars* __restrict__ sc, double* __restrict__ sigma_out) {
  __shared__ double S[kD * kD];
  __shared__ float Sf[kD * kD];  // Sigma rounded to float32 once, for the float32 work
  __shared__ double s_sum[kD * kD + kD + 1];

  const int tid = threadIdx.x;
  constexpr int kP = kD * kD + kD + 1;
  constexpr int kT = kD / 3;  // points of a patch: the pooled dimension
  // gather the moments
  double npd;
  if (dtype == 0) {
    for (int i = tid; i < kD * kD; i += kFinThreads) s_sum[i] = double(sc->s2[i]);
    for (int i = tid; i < kD; i += kFinThreads) s_sum[kD * kD + i] = double(sc->s1[i]);
    if (tid == 0) s_sum[kD * kD + kD] = double(sc->n_patches);
  } else {
    for (int i = tid; i < kP; i += kFinThreads) {
      double t = 0.0;
      for (int b = 0; b < nblocks; ++b) t += f64_partials[size_t(b) * kP + i];
      s_sum[i] = t;
    }
  }
  fin_bar();
  npd = s_sum[kD * kD + kD];
  if (tid == 0 && dtype == 1) sc->n_patches = (unsigned long long)npd;
  if (npd < 1.0) {
    if (tid < kD) sc->eig[tid] = 0.0;
    if (tid == 0) {
      sc->tau = 0.0;
      sc->sigma_est = 0.0;
      sc->m = 0;
      sc->ne_valid = 1;
      if (sigma_out) *sigma_out = 0.0;
      __threadfence();
      atomicExch(&sc->sigma_ready, 1u);
    }
    return;
  }
  if (!sc->pooled_patch) {
    // Sigma = S2/N - mu mu^T (upper triangle accumulated; mirror it)
    const double inv_n = 1.0 / npd;
    for (int e = tid; e < kD * kD; e += kFinThreads) {
      const int r = e / kD, c = e % kD;
      const int rr = min(r, c), cc = max(r, c);
      const double mr = s_sum[kD * kD + rr] * inv_n, mc = s_sum[kD * kD + cc] * inv_n;
      const double v = s_sum[rr * kD + cc] * inv_n - mr * mc;
      S[e] = v;
      Sf[e] = float(v);
    }
    fin_bar();
    eig_tail<kD>(S, Sf, sc, sigma_out, dtype);
    return;
  }
  // pooled: 3 N samples of kT entries; mu_i = sum_c s1[3i + c] / 3N,
  // Sigma_ij = sum_c s2[3i + c][3j + c] / 3N - mu_i mu_j
  const double inv_3n = 1.0 / (3.0 * npd);
  for (int e = tid; e < kT * kT; e += kFinThreads) {
    const int i = e / kT, j = e % kT;
    const int lo = min(i, j), hi = max(i, j);
    double s2 = 0.0, mi = 0.0, mj = 0.0;
    for (int c = 0; c < 3; ++c) {
      s2 += s_sum[(3 * lo + c) * kD + 3 * hi + c];
      mi += s_sum[kD * kD + 3 * i + c];
      mj += s_sum[kD * kD + 3 * j + c];
    }
    const double v = s2 * inv_3n - (mi * inv_3n) * (mj * inv_3n);
    S[e] = v;
    Sf[e] = float(v);
  }
  fin_bar();
  eig_tail<kT>(S, Sf, sc, sigma_out, dtype);
}

__global__ void __launch_bounds__(kFinThreads) k_ne_finalize(int dtype, const double* __restrict__ f64_partials,
                                                           int nblocks, DevScalars* __restrict__ sc,
                                                           double* __restrict__ sigma_out) {
  pdl_wait();
  finalize_block(dtype, f64_partials, nblocks, sc, sigma_out);
}

// One block per SM (the dynamic shared memory keeps a second one out): block 0
// computes sigma_est on an SM of its own, the others meanwhile take the first
// filter steps, which need the graph and the colours only.  With a.fuse they
// then also select and filter: they stop stepping once sigma_est is published
// (or after kSpecMax steps, then waiting for it) and run the selection over
// the stored steps (select_filter), so no second launch follows.
constexpr int kSpecThreads = 1024;
constexpr int kSpecPadBytes = 100 * 1024;  // shared memory that makes a second block not fit on an SM

// FUSE: the selection and filter follow in the same launch (a.fuse); a kernel
// of its own, so that the plain launch carries none of their registers.
template <bool FUSE>
__global__ void __launch_bounds__(kSpecThreads, 1)
    k_ne_finalize_spec(int dtype, const double* __restrict__ f64_partials, int nblocks, DevScalars* __restrict__ sc,
                       double* __restrict__ sigma_out, FilterArgs a) {
  pdl_wait();
  __shared__ int s_ok;
  __shared__ int s_go;
  __shared__ float s_cexp;
  if (blockIdx.x == 0) {
    if (threadIdx.x < kFinThreads) finalize_block(dtype, f64_partials, nblocks, sc, sigma_out);
    return;
  }
  uint32_t epoch = 0;
  const int S = speculative_steps(a, a.spec_depth, 1, gridDim.x - 1, FUSE, epoch, &s_ok, &s_cexp, &s_go);
  if (!FUSE || S < 0) return;
  // sigma_est of block 0 (a bounded wait)
  if (threadIdx.x == 0) {
    const unsigned long long t0 = global_ns();
    const unsigned long long limit = sc->wait_limit_ns;
    int ok = 1;
    while (!ld_acquire_u32(&sc->sigma_ready)) {
      if (global_ns() - t0 > limit) {
        atomicOr(&sc->status, kFlagTimeout);
        ok = 0;
        break;
      }
      __nanosleep(128);
    }
    s_ok = ok;
  }
  __syncthreads();
  if (!s_ok) return;
  select_filter<kSpecThreads>(a, S, 1, gridDim.x - 1, &sc->spec_barrier, epoch);
}

// Segmented estimate launch (one block per SM, cooperative): block f < count
// computes sigma_est of frame f, and frame f's share of the other blocks takes
// its speculative filter steps (no fused selection here).
struct EstimateSeg {
  FilterArgs spec[kSegMax];
  const double* f64_partials[kSegMax];
  int nblocks[kSegMax];
  int first[kSegMax + 1];  // frame f's step blocks: [count + first[f], count + first[f + 1])
  int count;
};

__global__ void __launch_bounds__(kSpecThreads, 1) k_ne_finalize_spec_seg(const __grid_constant__ EstimateSeg e) {
  pdl_wait();
  __shared__ int s_ok;
  __shared__ int s_go;
  __shared__ float s_cexp;
  if (int(blockIdx.x) < e.count) {
    const int f = blockIdx.x;
    if (threadIdx.x < kFinThreads) finalize_block(e.spec[f].dtype, e.f64_partials[f], e.nblocks[f], e.spec[f].sc, nullptr);
    return;
  }
  const int b = int(blockIdx.x) - e.count;
  int f = 0;
  while (f + 1 < e.count && e.first[f + 1] <= b) ++f;
  uint32_t epoch = 0;
  speculative_steps(e.spec[f], e.spec[f].spec_depth, e.count + e.first[f], uint32_t(e.first[f + 1] - e.first[f]),
                    false, epoch, &s_ok, &s_cexp, &s_go);
}

// testing: the float64 quotient of the eigen step beside CUDA's own division
__global__ void __launch_bounds__(256) k_debug_div(const double* __restrict__ a, const double* __restrict__ b,
                                                   double* __restrict__ q_newton, double* __restrict__ q_div,
                                                   int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    q_newton[i] = div_newton(a[i], b[i]);
    q_div[i] = a[i] / b[i];
  }
}

}  // namespace

cudaError_t launch_debug_div(const double* a, const double* b, double* q_newton, double* q_div, int64_t n,
                             cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = int(std::min<int64_t>((n + 255) / 256, 152 * 8));
  return launch_kernel(k_debug_div, dim3(grid), dim3(256), 0, stream, false, a, b, q_newton, q_div, n);
}

cudaError_t launch_gather_colors_seg(const GatherArgs* a, int count, cudaStream_t stream) {
  if (count < 1 || count > kSegMax) return cudaErrorInvalidValue;
  Seg<GatherArgs> sg;
  int blocks[kSegMax];
  for (int f = 0; f < count; ++f) {
    sg.a[f] = a[f];
    blocks[f] = a[f].n > 0 ? std::min((a[f].n + 1023) / 1024, 152 * 8) : 0;  // as launch_gather_colors
  }
  const int grid = seg_layout(sg, blocks, count);
  if (grid == 0) return cudaSuccess;
  return launch_kernel(k_gather_seg, dim3(grid), dim3(256), 0, stream, false, sg);
}

cudaError_t launch_ne_moments_seg(const MomentArgs* a, int count, int dtype, int num_sms, cudaStream_t stream) {
  if (count < 1 || count > kSegMax) return cudaErrorInvalidValue;
  Seg<MomentArgs> sg;
  int blocks[kSegMax];
  for (int f = 0; f < count; ++f) {
    sg.a[f] = a[f];
    blocks[f] = a[f].n > 0 ? ne_moment_blocks(a[f].n, num_sms) : 0;
  }
  const int grid = seg_layout(sg, blocks, count);
  if (grid == 0) return cudaSuccess;
  if (dtype == 0) return launch_kernel(k_ne_moments_seg<0>, dim3(grid), dim3(kNeThreads), 0, stream, false, sg);
  return launch_kernel(k_ne_moments_seg<1>, dim3(grid), dim3(kNeThreads), 0, stream, false, sg);
}

cudaError_t launch_ne_finalize_seg(const FilterArgs* spec, const double* const* f64_partials, const int* nblocks,
                                   int count, int num_sms, cudaStream_t stream) {
  if (count < 1 || count > kSegMax || num_sms < 2 * count) return cudaErrorInvalidValue;
  static std::atomic<unsigned long long> configured{0};  // the shared-memory limit is set once per device
  cudaError_t e = once_per_device(configured, [] {
    return cudaFuncSetAttribute(k_ne_finalize_spec_seg, cudaFuncAttributeMaxDynamicSharedMemorySize, kSpecPadBytes);
  });
  if (e != cudaSuccess) return e;
  EstimateSeg es;
  es.count = count;
  // the step blocks in proportion to the frames' points, at least one each
  const int pool = num_sms - count;
  double total = 0.0;
  for (int f = 0; f < count; ++f) total += double(std::max(spec[f].n, 1));
  int given = 0;
  es.first[0] = 0;
  for (int f = 0; f < count; ++f) {
    es.spec[f] = spec[f];
    es.f64_partials[f] = f64_partials[f];
    es.nblocks[f] = nblocks[f];
    const int left = count - 1 - f;  // frames after this one keep one block each
    int b = int(double(pool) * double(std::max(spec[f].n, 1)) / total);
    b = std::max(1, std::min(b, pool - given - left));
    if (f == count - 1) b = pool - given;
    given += b;
    es.first[f + 1] = given;
  }
  return launch_kernel(k_ne_finalize_spec_seg, dim3(count + pool), dim3(kSpecThreads), kSpecPadBytes, stream, true,
                       es);
}

cudaError_t launch_gather_colors(const void* rgb, int dtype, int n, const int32_t* perm1,
                                 uint32_t* y8, float4* yf, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = std::min((n + 1023) / 1024, 152 * 8);  // four points a thread
  if (dtype == 0)
    return launch_kernel(k_gather_u8, dim3(grid), dim3(256), 0, stream, false, static_cast<const uint8_t*>(rgb), n,
                         perm1, y8);
  return launch_kernel(k_gather_f32, dim3(grid), dim3(256), 0, stream, false, static_cast<const float*>(rgb), n,
                       perm1, yf);
}

int ne_moment_blocks(int n, int num_sms) {
  // resident blocks per SM, queried once (the same code runs on every device of one build)
  static const int per_sm = [] {
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_ne_moments<0>, kNeThreads, 0) != cudaSuccess || a < 1)
      a = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_ne_moments<1>, kNeThreads, 0) != cudaSuccess || b < 1)
      b = 1;
    cudaGetLastError();
    return std::min(a, b);
  }();
  return std::max(1, std::min((n + kNeThreads - 1) / kNeThreads, num_sms * per_sm));
}

MomentArgs moment_args(int n, int bits, const GraphBufs& gb, const uint32_t* y8, const float4* yf, float* spread,
                       double* f64_partials, bool moments, bool sorted_patches, DevScalars* sc) {
  return MomentArgs{n,  bits,         gb.pk, gb.c4, y8, yf, spread, f64_partials, moments ? 1 : 0, sorted_patches ? 1 : 0,
                    sc, nullptr};
}

cudaError_t launch_ne_moments(int n, int bits, int dtype, const GraphBufs& gb, const uint32_t* y8,
                              const float4* yf, float* spread, double* f64_partials,
                              DevScalars* sc, int num_sms, bool moments, bool sorted_patches,
                              cudaStream_t stream, float4* x0) {
  if (n <= 0) return cudaSuccess;
  const int grid = ne_moment_blocks(n, num_sms);
  MomentArgs a = moment_args(n, bits, gb, y8, yf, spread, f64_partials, moments, sorted_patches, sc);
  a.x0 = x0;
  if (dtype == 0) return launch_kernel(k_ne_moments<0>, dim3(grid), dim3(kNeThreads), 0, stream, false, a);
  return launch_kernel(k_ne_moments<1>, dim3(grid), dim3(kNeThreads), 0, stream, false, a);
}

cudaError_t launch_ne_finalize(int dtype, const double* f64_partials, int nblocks, DevScalars* sc,
                               double* sigma_out, const FilterArgs* spec, int num_sms, cudaStream_t stream) {
  if (!spec || spec->spec_depth <= 0 || spec->n <= 0 || num_sms < 2)
    return launch_kernel(k_ne_finalize, dim3(1), dim3(kFinThreads), 0, stream, false, dtype, f64_partials, nblocks,
                         sc, sigma_out);
  static std::atomic<unsigned long long> configured{0};  // the shared-memory limit is set once per device
  const cudaError_t e = once_per_device(configured, [] {
    cudaError_t r = cudaFuncSetAttribute(k_ne_finalize_spec<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kSpecPadBytes);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(k_ne_finalize_spec<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSpecPadBytes);
    return r;
  });
  if (e != cudaSuccess) return e;
  if (spec->fuse)
    return launch_kernel(k_ne_finalize_spec<true>, dim3(num_sms), dim3(kSpecThreads), kSpecPadBytes, stream, true,
                         dtype, f64_partials, nblocks, sc, sigma_out, *spec);
  return launch_kernel(k_ne_finalize_spec<false>, dim3(num_sms), dim3(kSpecThreads), kSpecPadBytes, stream, true,
                       dtype, f64_partials, nblocks, sc, sigma_out, *spec);
}

}  // namespace fgbd
