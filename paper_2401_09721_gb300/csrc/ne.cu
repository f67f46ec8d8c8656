// NE-GBP: noise estimation using graph-based patches (Section 2.3), plus the
// per-point colour spread that the limited region of FSLR uses (Section 2.4).
//
// k_gather_colors: colours of the caller (input order) into sorted order.
// k_ne_moments: per point, its patch {i} + neighbours.  The spread
//   (sigma_R + sigma_G + sigma_B)/3 is written for every point.  A point with
//   exactly 6 neighbours contributes the patch a_i = [f_i, f_n1, ..., f_n6],
//   neighbours in increasing distance (ties by offset (dz, dy, dx), then
//   index), to the first and second moments sum a and sum a a^T.  uint8
//   colours are centred on 128 and kept as int8, so the moments are exact
//   integer sums (dp4a over 4 patches per instruction, int64 accumulation).
// k_ne_finalize: one block.  Sigma = S2/N - mu mu^T in float64; a cyclic
//   Jacobi in float32 (parallel round-robin order) gives approximate
//   eigenvectors; each eigenvalue is then the float64 Rayleigh quotient
//   v^T Sigma v / v^T v, whose error is second order in the eigenvector error;
//   the values are sorted descending and the tail rule gives sigma_est.
#include <algorithm>

#include "fgbd_internal.cuh"

namespace fgbd {
namespace {

constexpr int kTiles = 28;  // 3x3 output tiles covering the upper triangle of a 21x21 matrix

__global__ void __launch_bounds__(256) k_gather_u8(const uint8_t* __restrict__ rgb, int n,
                                                   const int32_t* __restrict__ perm1,
                                                   uint32_t* __restrict__ y8) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int pi = perm1[k];
    if (!in_range(pi, n)) continue;
    const size_t i = size_t(pi);
    y8[k] = uint32_t(rgb[3 * i]) | (uint32_t(rgb[3 * i + 1]) << 8) | (uint32_t(rgb[3 * i + 2]) << 16);
  }
}

__global__ void __launch_bounds__(256) k_gather_f32(const float* __restrict__ rgb, int n,
                                                    const int32_t* __restrict__ perm1,
                                                    float4* __restrict__ yf) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int pi = perm1[k];
    if (!in_range(pi, n)) continue;
    const size_t i = size_t(pi);
    yf[k] = make_float4(rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], 0.f);
  }
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

template <int DT>
__device__ __forceinline__ void cswap(NbKey<DT>& a, NbKey<DT>& b) {
  const bool sw = (b.key < a.key) || (b.key == a.key && b.idx < a.idx);
  if (sw) {
    const NbKey<DT> t = a;
    a = b;
    b = t;
  }
}

constexpr int kNeWarps = kNeThreads / 32;
constexpr int kRowWords = 9;    // 32 int8 patch entries = 8 words, padded: the 21 rows start in distinct banks
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
                                            bool moments, uint8_t* at8, float* atf) {
  int nb[6];
  bool v[6];
  nb[0] = k - 1;
  v[0] = k > 0;
  nb[1] = k + 1;
  v[1] = k + 1 < n;
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
    const int nn = deg + 1;
    const float vr = float(nn * qr - sr * sr), vg = float(nn * qg - sg * sg), vb = float(nn * qb - sb * sb);
    sp = (sqrtf(vr) / cnt + sqrtf(vg) / cnt + sqrtf(vb) / cnt) / 3.0f;
  } else {
    const float4 o = yf[k];
    ownr = o.x;
    owng = o.y;
    ownb = o.z;
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
    mr /= cnt;
    mg /= cnt;
    mb /= cnt;
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
    sp = (sqrtf(vr / cnt) + sqrtf(vg / cnt) + sqrtf(vb / cnt)) / 3.0f;
  }
  spread[k] = sp;
  if (!patch) return false;

  int kx, ky, kz;
  decode_c1(pk[k], bits, kx, ky, kz);
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    int x, y, z;
    decode_c1(cpk[j], bits, x, y, z);
    const int dx = x - kx, dy = y - ky, dz = z - kz;
    const unsigned long long d2 = (unsigned long long)(dx * dx + dy * dy + dz * dz);
    e[j].key = (d2 << 33) | ((unsigned long long)(dz + 1024) << 22) | ((unsigned long long)(dy + 1024) << 11) |
               (unsigned long long)(dx + 1024);
  }
  // odd-even transposition sort, 6 rounds
#pragma unroll
  for (int round = 0; round < 6; ++round) {
    if ((round & 1) == 0) {
      cswap(e[0], e[1]);
      cswap(e[2], e[3]);
      cswap(e[4], e[5]);
    } else {
      cswap(e[1], e[2]);
      cswap(e[3], e[4]);
    }
  }
  if (DT == 0) {
    // entry r of the patch, centred on 128: the colour byte with its top bit flipped, read as int8
    const int stride = kRowWords * 4;
    at8[0 * stride + lane] = uint8_t((own8 & 255u) ^ 0x80u);
    at8[1 * stride + lane] = uint8_t(((own8 >> 8) & 255u) ^ 0x80u);
    at8[2 * stride + lane] = uint8_t(((own8 >> 16) & 255u) ^ 0x80u);
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const uint32_t c = reinterpret_cast<NbKey<0>&>(e[j]).col;
      at8[(3 + 3 * j) * stride + lane] = uint8_t((c & 255u) ^ 0x80u);
      at8[(4 + 3 * j) * stride + lane] = uint8_t(((c >> 8) & 255u) ^ 0x80u);
      at8[(5 + 3 * j) * stride + lane] = uint8_t(((c >> 16) & 255u) ^ 0x80u);
    }
  } else {
    atf[0 * kRowFloats + lane] = ownr - 128.f;
    atf[1 * kRowFloats + lane] = owng - 128.f;
    atf[2 * kRowFloats + lane] = ownb - 128.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const NbKey<1>& f = reinterpret_cast<NbKey<1>&>(e[j]);
      atf[(3 + 3 * j) * kRowFloats + lane] = f.r - 128.f;
      atf[(4 + 3 * j) * kRowFloats + lane] = f.g - 128.f;
      atf[(5 + 3 * j) * kRowFloats + lane] = f.b - 128.f;
    }
  }
  return true;
}

// Warp-synchronous: each warp takes 32 points at a time, stages their patches
// transposed in its own shared-memory block and accumulates the moments with
// __syncwarp only.  Lanes 0..27 own one 3x3 tile of the upper triangle of
// sum a a^T; lanes 28..31 own rows of sum a.  uint8 colours: exact int32 dp4a
// sums, moved to int64 every 1024 batches; float colours: fp32 sums over 4
// batches, then float64.  The block combines its warps through shared atomics
// and adds its totals to the context (uint8) or writes them (float).
template <int DT>
__global__ void __launch_bounds__(kNeThreads)
    k_ne_moments(int n, int bits, const uint32_t* __restrict__ pk, const int4* __restrict__ c4,
                 const uint32_t* __restrict__ y8, const float4* __restrict__ yf,
                 float* __restrict__ spread, double* __restrict__ f64_partials, int moments,
                 DevScalars* __restrict__ sc) {
  constexpr int kP = kD * kD + kD + 1;
  __shared__ __align__(16) uint32_t s_at8[DT == 0 ? kNeWarps : 1][kD * kRowWords];
  __shared__ __align__(16) float s_atf[DT == 1 ? kNeWarps : 1][kD * kRowFloats];
  __shared__ unsigned long long s_tot8[DT == 0 ? kP : 1];
  __shared__ double s_totf[DT == 1 ? kP : 1];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (moments) {
    for (int i = threadIdx.x; i < kP; i += kNeThreads) {
      if (DT == 0) s_tot8[i] = 0ull;
      else s_totf[i] = 0.0;
    }
  }
  __syncthreads();
  int r0 = 0, c0 = 0, rb = 0, re = 0;
  if (lane < kTiles) {
    tile_rc(lane, r0, c0);
  } else {
    rb = ((lane - kTiles) * kD) / kFirstLanes;
    re = ((lane - kTiles + 1) * kD) / kFirstLanes;
  }
  int acc[9] = {};
  long long acc64[9] = {};
  float accf[9] = {};
  double accd[9] = {};
  unsigned long long npatch = 0;
  int since_flush = 0;
  uint8_t* at8 = reinterpret_cast<uint8_t*>(&s_at8[DT == 0 ? warp : 0][0]);
  float* atf = &s_atf[DT == 1 ? warp : 0][0];

  const int nwarps = gridDim.x * kNeWarps;
  for (int base = (blockIdx.x * kNeWarps + warp) * 32; base < n; base += nwarps * 32) {
    const int k = base + lane;
    bool has = false;
    if (k < n) has = point_patch<DT>(k, n, bits, lane, pk, c4, y8, yf, spread, moments != 0, at8, atf);
    if (!moments) continue;
    if (!has) {
#pragma unroll
      for (int r = 0; r < kD; ++r) {
        if (DT == 0) at8[r * kRowWords * 4 + lane] = 0;
        else atf[r * kRowFloats + lane] = 0.f;
      }
    }
    const uint32_t hb = __ballot_sync(0xffffffffu, has);
    npatch += __popc(hb);
    __syncwarp();
    if (DT == 0) {
      const int* at = reinterpret_cast<const int*>(&s_at8[warp][0]);
      if (lane < kTiles) {
#pragma unroll
        for (int w = 0; w < 8; ++w) {
          int a[3], b[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            a[i] = at[(r0 + i) * kRowWords + w];
            b[i] = at[(c0 + i) * kRowWords + w];
          }
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) acc[3 * i + j] = __dp4a(a[i], b[j], acc[3 * i + j]);
        }
      } else {
#pragma unroll
        for (int t = 0; t < 6; ++t) {
          const int r = rb + t;
          if (r < re) {
#pragma unroll
            for (int w = 0; w < 8; ++w) acc[t] = __dp4a(at[r * kRowWords + w], 0x01010101, acc[t]);
          }
        }
      }
      if (++since_flush == 1024) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          acc64[i] += acc[i];
          acc[i] = 0;
        }
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
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    acc64[i] += acc[i];
    accd[i] += double(accf[i]);
  }
  // combine the warps of the block
  if (lane < kTiles) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const int idx = (r0 + i) * kD + (c0 + j);
        if (DT == 0) atomicAdd(&s_tot8[idx], (unsigned long long)acc64[3 * i + j]);
        else atomicAdd(&s_totf[idx], accd[3 * i + j]);
      }
  } else {
#pragma unroll
    for (int t = 0; t < 6; ++t) {
      const int r = rb + t;
      if (r < re) {
        if (DT == 0) atomicAdd(&s_tot8[kD * kD + r], (unsigned long long)acc64[t]);
        else atomicAdd(&s_totf[kD * kD + r], accd[t]);
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
      f64_partials[size_t(blockIdx.x) * kP + i] = s_totf[i];
    }
  }
}

// ---------------------------------------------------------------- finalize

constexpr double kZeroEigRel = 1e-9;  // relative size below which an eigenvalue is zero
constexpr int kMaxSweeps = 15;
constexpr int kFinThreads = 448;      // 14 warps: one thread per element of the 21 x 21 matrix

// Parallel cyclic Jacobi schedule on 21 indices: in round r (0..20) index i is
// paired with (2r - i) mod 21, and index r, which pairs with itself, rests.
// Every pair {i, j} meets exactly once per sweep, in the round r with
// 2r = i + j (mod 21).
__device__ __forceinline__ int jacobi_partner(int i, int r) {
  int p = 2 * r - i;
  if (p < 0) p += kD;
  if (p >= kD) p -= kD;
  return p;
}

// The rotation of round r acting on index x: new row/column x = alpha * old x +
// beta * old partner.  For the pair p < q with a_pq above the threshold the
// angle zeroes a_pq: cos 2phi = |a_qq - a_pp| / r, r = sqrt((a_qq - a_pp)^2 +
// 4 a_pq^2), c = sqrt((1 + cos 2phi) / 2), |s| = |a_pq| / (r c), and s takes
// the sign of (a_qq - a_pp) a_pq (the smaller of the two angles that zero it).
// Every thread derives the coefficients from the same three entries with the
// same operations, so all threads agree on them bit for bit.
__device__ __forceinline__ bool jacobi_coef(const float* __restrict__ A, int x, int px, float thr, float& alpha,
                                            float& beta) {
  alpha = 1.f;
  beta = 0.f;
  if (px == x) return false;
  const int p = min(x, px), q = max(x, px);
  const float apq = A[p * kD + q];
  if (!(fabsf(apq) > thr)) return false;
  const float tau = A[q * kD + q] - A[p * kD + p];
  const float two_a = 2.f * apq;
  const float rr = rsqrtf(fmaf(tau, tau, two_a * two_a));
  const float h = fmaf(0.5f * fabsf(tau), rr, 0.5f);
  const float ic = rsqrtf(h);
  const float c = h * ic;
  float s = fabsf(apq) * rr * ic;
  if ((tau < 0.f) != (apq < 0.f)) s = -s;
  alpha = c;
  beta = (x == p) ? -s : s;
  return true;
}

__global__ void __launch_bounds__(kFinThreads) k_ne_finalize(int dtype, const double* __restrict__ f64_partials,
                                                     int nblocks, DevScalars* __restrict__ sc,
                                                     double* __restrict__ sigma_out) {
  __shared__ double S[kD][kD];
  __shared__ double s_sum[kD * kD + kD + 1];
  __shared__ float V[kD][kD + 1];
  __shared__ float Abuf[2][kD * kD];
  __shared__ float Vbuf[2][kD * kD];
  __shared__ double s_lam[kD];
  __shared__ double s_sorted[kD];
  __shared__ double s_num[kD][kD];
  __shared__ double V64[kD][kD + 1];
  __shared__ double s_suffix[kD + 1];
  __shared__ int s_pass;

  const int tid = threadIdx.x;
  constexpr int kP = kD * kD + kD + 1;
  // gather the moments
  double npd;
  if (dtype == 0) {
    for (int i = tid; i < kD * kD; i += blockDim.x) s_sum[i] = double(sc->s2[i]);
    for (int i = tid; i < kD; i += blockDim.x) s_sum[kD * kD + i] = double(sc->s1[i]);
    if (tid == 0) s_sum[kD * kD + kD] = double(sc->n_patches);
  } else {
    for (int i = tid; i < kP; i += blockDim.x) {
      double t = 0.0;
      for (int b = 0; b < nblocks; ++b) t += f64_partials[size_t(b) * kP + i];
      s_sum[i] = t;
    }
  }
  __syncthreads();
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
    }
    return;
  }
  // Sigma = S2/N - mu mu^T (upper triangle accumulated; mirror it)
  const double inv_n = 1.0 / npd;
  for (int e = tid; e < kD * kD; e += blockDim.x) {
    const int r = e / kD, c = e % kD;
    const int rr = min(r, c), cc = max(r, c);
    const double mr = s_sum[kD * kD + rr] * inv_n, mc = s_sum[kD * kD + cc] * inv_n;
    S[r][c] = s_sum[rr * kD + cc] * inv_n - mr * mc;
  }
  __syncthreads();

  // Cyclic Jacobi in float32 over the whole block, matrix and vectors in
  // shared memory (double-buffered), thread t < 441 owning entry (t / 21,
  // t % 21) of A and of V.  One barrier per round: each thread derives the
  // rotations of its row and column indices itself.  A pair is rotated only
  // while |a_pq| > 2e-7 ||diag A|| (the float32 resolution of the matrix); the
  // iteration ends at the first barrier where no off-diagonal entry is above
  // that threshold, since no later round would rotate anything.
  {
    const bool owner = tid < kD * kD;
    const int ei = owner ? tid / kD : 0, ej = owner ? tid % kD : 0;
    const int lo = min(ei, ej), hi = max(ei, ej);
    if (owner) {
      Abuf[0][tid] = float(S[ei][ej]);
      Vbuf[0][tid] = ei == ej ? 1.f : 0.f;
    }
    float dsq = 0.f;
    for (int i = 0; i < kD; ++i) dsq = fmaf(float(S[i][i]), float(S[i][i]), dsq);
    const float thr = 2e-7f * sqrtf(dsq);
    int cur = 0;
    bool big = __syncthreads_or(owner && ei != ej && fabsf(Abuf[0][tid]) > thr);
    for (int round = 0; big && round < kMaxSweeps * kD; ++round) {
      const int r = round % kD;
      const float* A = Abuf[cur];
      const float* Vc = Vbuf[cur];
      bool off_big = false;
      if (owner) {
        // A' = J^T A J evaluated for (lo, hi) so that both mirror entries get the same bits
        const int plo = jacobi_partner(lo, r), phi = jacobi_partner(hi, r);
        float al, bl, ah, bh;
        jacobi_coef(A, lo, plo, thr, al, bl);
        jacobi_coef(A, hi, phi, thr, ah, bh);
        const float row_lo = fmaf(ah, A[lo * kD + hi], bh * A[lo * kD + phi]);
        const float row_plo = fmaf(ah, A[plo * kD + hi], bh * A[plo * kD + phi]);
        const float a = fmaf(al, row_lo, bl * row_plo);
        // V' = V J: column ej of row ei, with the coefficients of index ej
        const bool j_lo = ej == lo;
        const float aj = j_lo ? al : ah, bj = j_lo ? bl : bh;
        const int pj = j_lo ? plo : phi;
        Abuf[cur ^ 1][tid] = a;
        Vbuf[cur ^ 1][tid] = fmaf(aj, Vc[ei * kD + ej], bj * Vc[ei * kD + pj]);
        off_big = ei != ej && fabsf(a) > thr;
      }
      cur ^= 1;
      big = __syncthreads_or(off_big);
    }
    if (owner) V[ei][ej] = Vbuf[cur][tid];
  }
  __syncthreads();

  // float64 Rayleigh quotients of the 21 eigenvector estimates
  for (int e = tid; e < kD * kD; e += blockDim.x) V64[e / kD][e % kD] = double(V[e / kD][e % kD]);
  __syncthreads();
  for (int e = tid; e < kD * kD; e += blockDim.x) {
    const int k = e / kD, r = e % kD;
    double w = 0.0;
#pragma unroll 7
    for (int c = 0; c < kD; ++c) w = fma(S[r][c], V64[c][k], w);
    s_num[k][r] = w * V64[r][k];
  }
  __syncthreads();
  if (tid < kD) {
    double num = 0.0, den = 0.0;
    for (int r = 0; r < kD; ++r) {
      num += s_num[tid][r];
      den = fma(V64[r][tid], V64[r][tid], den);
    }
    s_lam[tid] = num / den;
  }
  __syncthreads();
  // eigenvalues below 1e-9 max(lambda_1, 1) are numerical zeros (a rank-deficient
  // covariance); they are set to exactly 0 so the tail rule never decides on rounding noise
  if (tid < kD) {
    double top = s_lam[0];
    for (int j = 1; j < kD; ++j) top = fmax(top, s_lam[j]);
    const double l = s_lam[tid];
    const bool zero = fabs(l) < kZeroEigRel * fmax(top, 1.0);
    __syncwarp(0x1fffffu);
    if (zero) s_lam[tid] = 0.0;
  }
  __syncthreads();
  if (tid < kD) {
    const double l = s_lam[tid];
    int rank = 0;
    for (int j = 0; j < kD; ++j) {
      const double o = s_lam[j];
      rank += (o > l) || (o == l && j < tid);
    }
    s_sorted[rank] = l;
  }
  __syncthreads();
  if (tid < kD) sc->eig[tid] = s_sorted[tid];
  // tail sums, accumulated from the smallest eigenvalue up so that a tail of
  // exact zeros sums to exactly 0
  if (tid == 0) {
    s_suffix[kD] = 0.0;
    for (int i = kD - 1; i >= 0; --i) s_suffix[i] = s_suffix[i + 1] + s_sorted[i];
  }
  __syncthreads();
  // tail rule, every m tested at once: the smallest m with
  // mean(lambda_{m+1..D}) <= median(lambda_{m+1..D}); m = D - 1 always passes
  if (tid < 32) {
    bool pass = false;
    double mean = 0.0;
    if (tid < kD) {
      const int cnt = kD - tid;
      mean = s_suffix[tid] / double(cnt);
      const double med = (cnt & 1) ? s_sorted[tid + cnt / 2]
                                   : 0.5 * (s_sorted[tid + cnt / 2 - 1] + s_sorted[tid + cnt / 2]);
      pass = mean <= med;
    }
    const unsigned passing = __ballot_sync(0xffffffffu, pass);
    const int m = __ffs(passing) - 1;
    if (tid == m) s_pass = m;
  }
  __syncthreads();
  if (tid == 0) {
    const int m = s_pass;
    const double tau = s_suffix[m] / double(kD - m);
    const double sg = sqrt(fmax(tau, 0.0));
    sc->m = m;
    sc->tau = tau;
    sc->sigma_est = sg;
    sc->ne_valid = 1;
    if (sigma_out) *sigma_out = sg;
  }
}

}  // namespace

cudaError_t launch_gather_colors(const void* rgb, int dtype, int n, const int32_t* perm1,
                                 uint32_t* y8, float4* yf, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = std::min((n + 255) / 256, 152 * 16);
  if (dtype == 0)
    k_gather_u8<<<grid, 256, 0, stream>>>(static_cast<const uint8_t*>(rgb), n, perm1, y8);
  else
    k_gather_f32<<<grid, 256, 0, stream>>>(static_cast<const float*>(rgb), n, perm1, yf);
  return cudaGetLastError();
}

int ne_moment_blocks(int n, int num_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ne_moments<0>, kNeThreads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  int per_sm_f = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_f, k_ne_moments<1>, kNeThreads, 0) != cudaSuccess ||
      per_sm_f < 1)
    per_sm_f = 1;
  per_sm = std::min(per_sm, per_sm_f);
  return std::max(1, std::min((n + kNeThreads - 1) / kNeThreads, num_sms * per_sm));
}

cudaError_t launch_ne_moments(int n, int bits, int dtype, const GraphBufs& gb, const uint32_t* y8,
                              const float4* yf, float* spread, double* f64_partials,
                              DevScalars* sc, int num_sms, bool moments, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  const int grid = ne_moment_blocks(n, num_sms);
  if (dtype == 0)
    k_ne_moments<0><<<grid, kNeThreads, 0, stream>>>(n, bits, gb.pk, gb.c4, y8, yf, spread, f64_partials,
                                                     moments ? 1 : 0, sc);
  else
    k_ne_moments<1><<<grid, kNeThreads, 0, stream>>>(n, bits, gb.pk, gb.c4, y8, yf, spread, f64_partials,
                                                     moments ? 1 : 0, sc);
  return cudaGetLastError();
}

cudaError_t launch_ne_finalize(int dtype, const double* f64_partials, int nblocks, DevScalars* sc,
                               double* sigma_out, cudaStream_t stream) {
  k_ne_finalize<<<1, kFinThreads, 0, stream>>>(dtype, f64_partials, nblocks, sc, sigma_out);
  return cudaGetLastError();
}

}  // namespace fgbd
