// NE-GBP (Section 2.3) at windows w > 1.  With w points linked on each side
// along each of the three codes (Section 2.2), a point has up to K = 6w
// neighbours, and the points with exactly K give patches of D = 3 (K + 1)
// entries: the point, then its neighbours by increasing distance (ties by the
// offset (dz, dy, dx), then by index), three colour channels each.  The FSLR
// spread of every point (Section 2.4) comes from the same pass.  Four launches:
//
//   k_ne_moments_wide  batches of points staged as a transposed patch block in
//                      shared memory; each thread owns one 3x3 tile (node a,
//                      node b >= a) of sum a a^T or the three sums a of one
//                      node.  uint8 colours: int8 entries c - 128 and exact
//                      dp4a sums in int64; float colours: float32 sums per
//                      batch, then float64.  Each block writes its partial
//                      sums (no atomics, so the totals do not depend on timing).
//   k_ne_wide_reduce   the partials summed entry by entry in a fixed order.
//   k_ne_wide_eigvec   one block: Sigma = S2/N - mu mu^T in float64, then
//                      float32 eigenvector estimates by a Householder
//                      tridiagonalisation, Sturm multisection and inverse
//                      iteration (tridiag.cuh).
//   k_ne_wide_tail     one block per eigenvector: the float64 Rayleigh quotient
//                      v^T Sigma v / v^T v (second order in the eigenvector
//                      error); the last block to finish sorts the values, sets
//                      numerical zeros to 0 and applies the tail rule.
#include <algorithm>
#include <atomic>

#include "eigen.cuh"
#include "gram_mma.cuh"
#include "tridiag.cuh"

namespace fgbd {
namespace {

constexpr int kWThreads = 256;        // moments: threads per block
constexpr int kWEigThreads = 256;   // the eigenvector block (255 registers a thread: the reducing warp holds two rows of A a lane)
constexpr int kWTailThreads = 64;     // D <= 57 eigenvector entries, one per thread

template <int W>
constexpr int patch_dim() {
  return 3 * (6 * W + 1);
}

// compare-exchange of two (key, sorted id) pairs: ascending key, then id
__device__ __forceinline__ void cmp_swap(unsigned long long& ka, int& ia, unsigned long long& kb, int& ib) {
  const bool sw = (kb < ka) || (kb == ka && ib < ia);
  const unsigned long long k0 = sw ? kb : ka, k1 = sw ? ka : kb;
  const int i0 = sw ? ib : ia, i1 = sw ? ia : ib;
  ka = k0;
  kb = k1;
  ia = i0;
  ib = i1;
}

// Sorted point k: its FSLR spread over itself and all its neighbours
// (spread[k]) and, if it has exactly K = 6W neighbours, its patch written to
// column `col` of the transposed batch block `rows` (row stride `rw`
// elements; uint8: float16 entries c - 128, exact; float: float c - 128).
// Returns whether a patch was written.
template <int W, int DT>
__device__ __forceinline__ bool wide_patch(int k, int n, int bits, const GraphBufs& gb, const uint32_t* __restrict__ y8,
                                           const float4* __restrict__ yf, float* __restrict__ spread, int col,
                                           uint32_t* rows, int rw) {
  constexpr int K = 6 * W;
  const uint32_t pkk = gb.pk[k];
  const int4 s = gb.c4[k];
  int id[K];
  int deg = 0;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    id[j] = neighbour_of(j, k, n, pkk, s, gb.cx, gb.cx_stride);
    deg += id[j] >= 0;
  }
  const int nn = deg + 1;
  float sp;
  if (DT == 0) {
    const uint32_t own = y8[k];
    int sr = int(own & 255u), sg = int((own >> 8) & 255u), sb = int((own >> 16) & 255u);
    int qr = sr * sr, qg = sg * sg, qb = sb * sb;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (id[j] < 0) continue;
      const uint32_t c = y8[id[j]];
      const int a = int(c & 255u), b = int((c >> 8) & 255u), d = int((c >> 16) & 255u);
      sr += a;
      sg += b;
      sb += d;
      qr += a * a;
      qg += b * b;
      qb += d * d;
    }
    // nn^2 times each population variance is an exact integer (as at window 1)
    const float vr = float(nn * qr - sr * sr), vg = float(nn * qg - sg * sg), vb = float(nn * qb - sb * sb);
    sp = (sqrtf(vr) + sqrtf(vg) + sqrtf(vb)) * __frcp_rn(3.0f * float(nn));
  } else {
    const float4 o = yf[k];
    float mr = o.x, mg = o.y, mb = o.z;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (id[j] < 0) continue;
      const float4 c = yf[id[j]];
      mr += c.x;
      mg += c.y;
      mb += c.z;
    }
    const float icnt = __frcp_rn(float(nn));
    mr *= icnt;
    mg *= icnt;
    mb *= icnt;
    float vr = (o.x - mr) * (o.x - mr), vg = (o.y - mg) * (o.y - mg), vb = (o.z - mb) * (o.z - mb);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (id[j] < 0) continue;
      const float4 c = yf[id[j]];
      vr += (c.x - mr) * (c.x - mr);
      vg += (c.y - mg) * (c.y - mg);
      vb += (c.z - mb) * (c.z - mb);
    }
    sp = (sqrtf(vr * icnt) + sqrtf(vg * icnt) + sqrtf(vb * icnt)) * (1.0f / 3.0f);
  }
  spread[k] = sp;
  if (deg != K) return false;

  // sort keys: d^2, then the offset (dz, dy, dx), packed so that integer order is lexicographic
  int kx, ky, kz;
  decode_c1(pkk, bits, kx, ky, kz);
  unsigned long long key[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    int x, y, z;
    decode_c1(gb.pk[id[j]], bits, x, y, z);
    const int dx = x - kx, dy = y - ky, dz = z - kz;
    const unsigned long long d2 = (unsigned long long)(dx * dx + dy * dy + dz * dz);
    key[j] = (d2 << 33) | ((unsigned long long)(dz + 1024) << 22) | ((unsigned long long)(dy + 1024) << 11) |
             (unsigned long long)(dx + 1024);
  }
  // Batcher's odd-even merge sort for K elements (42 comparators at K = 12,
  // 90 at K = 18, against K (K - 1) / 2 of a transposition sort); the keys
  // with their id are a strict order, so any sorting network gives the unique
  // sorted result.  All bounds are compile-time, so the network unrolls into
  // straight compare-exchanges on registers.
#pragma unroll
  for (int p = 1; p < K; p <<= 1) {
#pragma unroll
    for (int kk = p; kk >= 1; kk >>= 1) {
#pragma unroll
      for (int j = kk % p; j + kk < K; j += 2 * kk) {
#pragma unroll
        for (int i = 0; i < kk && i + j + kk < K; ++i) {
          if ((i + j) / (2 * p) == (i + j + kk) / (2 * p))
            cmp_swap(key[i + j], id[i + j], key[i + j + kk], id[i + j + kk]);
        }
      }
    }
  }
  if (DT == 0) {
    __half* h = reinterpret_cast<__half*>(rows);
    const uint32_t own = y8[k];
    h[0 * rw + col] = __int2half_rn(int(own & 255u) - 128);
    h[1 * rw + col] = __int2half_rn(int((own >> 8) & 255u) - 128);
    h[2 * rw + col] = __int2half_rn(int((own >> 16) & 255u) - 128);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const uint32_t c = y8[id[j]];
      h[(3 + 3 * j) * rw + col] = __int2half_rn(int(c & 255u) - 128);
      h[(4 + 3 * j) * rw + col] = __int2half_rn(int((c >> 8) & 255u) - 128);
      h[(5 + 3 * j) * rw + col] = __int2half_rn(int((c >> 16) & 255u) - 128);
    }
  } else {
    float* f = reinterpret_cast<float*>(rows);
    const float4 own = yf[k];
    f[0 * rw + col] = own.x - 128.f;
    f[1 * rw + col] = own.y - 128.f;
    f[2 * rw + col] = own.z - 128.f;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const float4 c = yf[id[j]];
      f[(3 + 3 * j) * rw + col] = c.x - 128.f;
      f[(4 + 3 * j) * rw + col] = c.y - 128.f;
      f[(5 + 3 * j) * rw + col] = c.z - 128.f;
    }
  }
  return true;
}

// uint8 colours, per block: batches of B = 256 points, one per thread, staged
// as float16 entry-major rows (entries, then the constant 1 of each valid
// patch, then zero rows up to a multiple of 16); the upper triangle of the
// Gram matrix of (a, 1) is covered by 16 x 8 blocks (mt, nt) with nt >= 2 mt,
// shared out among the warps, each summed over the batch by mma.sync
// (gram_mma.cuh) and moved to exact int64 sums in shared memory after every
// batch.  The block's sums go to part[blockIdx.x][D*D + D + 1] as int64 bit
// patterns (second moments at r*D + c, r <= c, 0 below the diagonal; first
// moments at D*D + r; the patch count last).
constexpr int kWBatch = 256;          // patches of a batch: one per thread
constexpr int kWHRow = kWBatch + 8;   // halves a staged row (528-byte rows: ldmatrix rows in distinct banks)

template <int W>
struct WideGram {
  static constexpr int D = patch_dim<W>();
  static constexpr int De = D + 1;             // with the constant entry
  static constexpr int MT = (De + 15) / 16;    // 16-row blocks
  static constexpr int NTL = (De + 7) / 8;     // 8-column blocks holding entries
  static constexpr int Tiles = [] {
    int c = 0;
    for (int mt = 0; mt < MT; ++mt) c += NTL - 2 * mt > 0 ? NTL - 2 * mt : 0;
    return c;
  }();
  static constexpr int PerWarp = (Tiles + kWThreads / 32 - 1) / (kWThreads / 32);
  static constexpr size_t RowBytes = size_t(16 * MT) * kWHRow * 2;
  static constexpr size_t SmemBytes = RowBytes + size_t(D * D + D) * 8;
  static_assert(kWBatch == kWThreads, "one patch per thread");
  static_assert(2 * MT >= NTL, "every column block's B operand comes from a row block");
};

template <int W>
__global__ void __launch_bounds__(kWThreads) k_ne_moments_wide_tc(int n, int bits, GraphBufs gb,
                                                                  const uint32_t* __restrict__ y8,
                                                                  float* __restrict__ spread,
                                                                  double* __restrict__ part) {
  pdl_wait();
  using G = WideGram<W>;
  constexpr int D = G::D, P = D * D + D + 1;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __half* rows = reinterpret_cast<__half*>(s_dyn);
  unsigned long long* sums = reinterpret_cast<unsigned long long*>(s_dyn + G::RowBytes);  // s2, then s1
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < int(G::RowBytes / 4); i += kWThreads) reinterpret_cast<uint32_t*>(rows)[i] = 0u;
  for (int i = tid; i < D * D + D; i += kWThreads) sums[i] = 0ull;
  // this warp's blocks of the Gram matrix: tiles warp, warp + 8, ...
  int tm[G::PerWarp], tn[G::PerWarp];
#pragma unroll
  for (int j = 0; j < G::PerWarp; ++j) {
    int t = warp + j * (kWThreads / 32), mt = 0;
    tm[j] = -1;
    tn[j] = 0;
    if (t >= G::Tiles) continue;
    while (t >= G::NTL - 2 * mt) {
      t -= G::NTL - 2 * mt;
      ++mt;
    }
    tm[j] = mt;
    tn[j] = 2 * mt + t;
  }
  __syncthreads();
  const uint32_t hbase = uint32_t(__cvta_generic_to_shared(rows));
  unsigned long long npatch = 0;
  for (int base = blockIdx.x * kWBatch; base < n; base += gridDim.x * kWBatch) {
    const int k = base + tid;
    bool has = false;
    if (k < n) has = wide_patch<W, 0>(k, n, bits, gb, y8, nullptr, spread, tid, reinterpret_cast<uint32_t*>(rows),
                                      kWHRow);
    if (!has) {
#pragma unroll 3
      for (int r = 0; r < D; ++r) rows[r * kWHRow + tid] = __float2half_rn(0.f);
    }
    rows[D * kWHRow + tid] = __float2half_rn(has ? 1.f : 0.f);
    npatch += (unsigned long long)__syncthreads_count(has);
#pragma unroll
    for (int j = 0; j < G::PerWarp; ++j) {
      if (tm[j] < 0) continue;
      float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
      for (int ks = 0; ks < kWBatch / 16; ++ks) {
        uint32_t a[4], b[4];
        ldsm_x4(gram_tile_addr(hbase, 16 * tm[j], 16 * ks, kWHRow, lane), a);
        ldsm_x4(gram_tile_addr(hbase, 16 * (tn[j] >> 1), 16 * ks, kWHRow, lane), b);
        if (tn[j] & 1) mma_16816(c, a, b[1], b[3]);
        else mma_16816(c, a, b[0], b[2]);
      }
      static_assert(kWBatch <= kGramFlushPatches, "one batch per accumulator before the move to int64");
      gram_flush(c, tm[j], tn[j], G::De, lane, sums, sums + D * D);
    }
    __syncthreads();  // the rows are rewritten by the next batch
  }
  __syncthreads();
  long long* out = reinterpret_cast<long long*>(part + size_t(blockIdx.x) * P);
  for (int i = tid; i < D * D + D; i += kWThreads) out[i] = (long long)sums[i];
  if (tid == 0) out[D * D + D] = (long long)npatch;
}

// Float colours, per block: batches of B = 128 points, one per thread of the
// first B; each thread owns one 3x3 tile (node a, node b >= a) of sum a a^T or
// the three sums a of one node, in float32 per batch, then float64; partial
// sums to part[blockIdx.x][D*D + D + 1] (second moments at r*D + c for the
// computed tiles, first moments at D*D + r, the patch count last).
template <int W>
__global__ void __launch_bounds__(kWThreads) k_ne_moments_wide_f32(int n, int bits, GraphBufs gb,
                                                                   const float4* __restrict__ yf,
                                                                   float* __restrict__ spread,
                                                                   double* __restrict__ part) {
  pdl_wait();
  constexpr int T = 6 * W + 1;  // points of a patch
  constexpr int D = 3 * T;
  constexpr int B = 128;
  constexpr int RW = B + 1;                        // row stride in words, odd: rows start in distinct banks
  constexpr int NT = T * (T + 1) / 2;              // tiles (a, b), a <= b
  constexpr int P = D * D + D + 1;
  static_assert(NT + T <= kWThreads && B <= kWThreads, "one tile or one first-moment node per thread");
  static_assert(D * RW * 4 <= 48 * 1024, "the batch block fits static shared memory");
  __shared__ __align__(16) uint32_t rows[D * RW];

  const int tid = threadIdx.x;
  int ta = -1, tb = -1;  // tile (ta, tb), or the first moments of node ta (tb = -1)
  if (tid < NT) {
    int t = tid, a = 0;
    while (t >= T - a) {
      t -= T - a;
      ++a;
    }
    ta = a;
    tb = a + t;
  } else if (tid < NT + T) {
    ta = tid - NT;
  }
  double accd[9] = {};
  unsigned long long npatch = 0;
  for (int base = blockIdx.x * B; base < n; base += gridDim.x * B) {
    bool has = false;
    if (tid < B) {
      const int k = base + tid;
      if (k < n) has = wide_patch<W, 1>(k, n, bits, gb, nullptr, yf, spread, tid, rows, RW);
      if (!has) {
        float* f = reinterpret_cast<float*>(rows);
#pragma unroll 3
        for (int r = 0; r < D; ++r) f[r * RW + tid] = 0.f;
      }
    }
    npatch += (unsigned long long)__syncthreads_count(has);
    const float* rf = reinterpret_cast<const float*>(rows);
    if (tb >= 0) {
      float accf[9] = {};
#pragma unroll 4
      for (int p = 0; p < B; ++p) {
        float a[3], b[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          a[i] = rf[(3 * ta + i) * RW + p];
          b[i] = rf[(3 * tb + i) * RW + p];
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) accf[3 * i + j] = fmaf(a[i], b[j], accf[3 * i + j]);
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) accd[i] += double(accf[i]);
    } else if (ta >= 0) {
      float accf[3] = {};
#pragma unroll 4
      for (int p = 0; p < B; ++p)
#pragma unroll
        for (int i = 0; i < 3; ++i) accf[i] += rf[(3 * ta + i) * RW + p];
#pragma unroll
      for (int i = 0; i < 3; ++i) accd[i] += double(accf[i]);
    }
    __syncthreads();
  }
  double* out = part + size_t(blockIdx.x) * P;
  if (tb >= 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) out[(3 * ta + i) * D + 3 * tb + j] = accd[3 * i + j];
  } else if (ta >= 0) {
#pragma unroll
    for (int i = 0; i < 3; ++i) out[D * D + 3 * ta + i] = accd[i];
  }
  if (tid == 0) out[D * D + D] = double(npatch);
}

// The totals: block (32 entries) x 8 warps; warp w sums the partial rows
// w, w + 8, ... of its lane's entry, and the eight warp sums are added in warp
// order, so the result does not depend on timing.  Second moments outside the
// computed tiles (below the diagonal blocks) are 0.
constexpr int kReduceWarps = 8;

template <int DT>
__global__ void __launch_bounds__(32 * kReduceWarps) k_ne_wide_reduce(const double* __restrict__ part, int blocks,
                                                                      int D, double* __restrict__ tot) {
  pdl_wait();
  __shared__ double s_f[kReduceWarps][32];
  __shared__ long long s_i[kReduceWarps][32];
  const int P = D * D + D + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  const bool used = i < P && (i >= D * D || (i / D) / 3 <= (i % D) / 3);
  long long ti = 0;
  double tf = 0.0;
  if (used) {
    if (DT == 0) {
      const long long* pi = reinterpret_cast<const long long*>(part);
#pragma unroll 4
      for (int b = warp; b < blocks; b += kReduceWarps) ti += pi[size_t(b) * P + i];
    } else {
#pragma unroll 4
      for (int b = warp; b < blocks; b += kReduceWarps) tf += part[size_t(b) * P + i];
    }
  }
  s_i[warp][lane] = ti;
  s_f[warp][lane] = tf;
  __syncthreads();
  if (warp == 0 && i < P) {
    long long a = 0;
    double f = 0.0;
    for (int w = 0; w < kReduceWarps; ++w) {
      a += s_i[w][lane];
      f += s_f[w][lane];
    }
    tot[i] = DT == 0 ? double(a) : f;  // integer totals stay below 2^53 for any capacity: exact
  }
}

struct BlockBar {
  __device__ void operator()() const { __syncthreads(); }
};

template <int D>
constexpr size_t wide_eig_smem() {
  return (sizeof(TridiagSmem<D, kWEigThreads>) + 15) / 16 * 16 + size_t(D) * D * 4;
}

// One block: the covariance Sigma = S2/N - mu mu^T in float64 (to S), then
// float32 eigenvector estimates (tridiag.cuh) to Vout, row-major with the
// vectors as columns, followed by their D float32 eigenvalues (the fallback of
// a non-finite Rayleigh quotient).  Without patches the results are written
// here (zero).
template <int D>
__global__ void __launch_bounds__(kWEigThreads) k_ne_wide_eigvec(const double* __restrict__ tot,
                                                                 double* __restrict__ S, float* __restrict__ Vout,
                                                                 DevScalars* __restrict__ sc,
                                                                 double* __restrict__ sigma_out) {
  pdl_wait();
  extern __shared__ __align__(16) unsigned char s_dyn[];
  TridiagSmem<D, kWEigThreads>& tw = *reinterpret_cast<TridiagSmem<D, kWEigThreads>*>(s_dyn);
  float* Sf = reinterpret_cast<float*>(s_dyn + (sizeof(TridiagSmem<D, kWEigThreads>) + 15) / 16 * 16);
  const int tid = threadIdx.x;
  const double npd = tot[D * D + D];
  if (tid == 0) sc->n_patches = (unsigned long long)npd;
  if (!(npd >= 1.0)) {
    for (int i = tid; i < D; i += kWEigThreads) sc->eig[i] = 0.0;
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
  const double inv_n = 1.0 / npd;
  for (int e = tid; e < D * D; e += kWEigThreads) {
    const int r = e / D, c = e % D;
    const int rr = min(r, c), cc = max(r, c);
    const double mr = tot[D * D + rr] * inv_n, mc = tot[D * D + cc] * inv_n;
    const double v = tot[rr * D + cc] * inv_n - mr * mc;
    S[e] = v;
    Sf[e] = float(v);
  }
  __syncthreads();
  eig_vectors_f32<D, kWEigThreads>(Sf, tw, Vout, Vout + D * D, BlockBar{});
}

// Block k: lambda_k = v_k^T Sigma v_k / v_k^T v_k in float64.  The last block
// to finish (a counter; no block waits for another) sorts the D values
// descending, sets those below 1e-9 max(lambda_1, 1) to 0 and applies the tail
// rule: m* is the smallest m with mean(lambda_{m+1..D}) <= median(lambda_{m+1..D}),
// sigma_est = sqrt(tau(m*)).
template <int D>
__global__ void __launch_bounds__(kWTailThreads) k_ne_wide_tail(const double* __restrict__ tot,
                                                                const double* __restrict__ S,
                                                                const float* __restrict__ V,
                                                                double* __restrict__ lam, uint32_t* __restrict__ done,
                                                                DevScalars* __restrict__ sc,
                                                                double* __restrict__ sigma_out) {
  pdl_wait();
  static_assert(D <= kWTailThreads, "one eigenvalue per thread in the last block");
  __shared__ double s_v[D];
  __shared__ double s_red[2][2];
  __shared__ int s_last;
  __shared__ long long s_key[D];
  __shared__ double s_sorted[D];
  __shared__ double s_suffix[D];
  __shared__ double s_top[2];
  __shared__ int s_m;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (!(tot[D * D + D] >= 1.0)) return;  // no patches: the eigenvector launch wrote the results
  const int k = blockIdx.x;
  if (tid < D) s_v[tid] = double(V[tid * D + k]);
  __syncthreads();
  double num = 0.0, den = 0.0;
  if (tid < D) {
    const double* row = S + size_t(tid) * D;
    double u0 = 0.0, u1 = 0.0, u2 = 0.0;
#pragma unroll
    for (int c = 0; c < D; c += 3) {
      u0 = fma(row[c], s_v[c], u0);
      u1 = fma(row[c + 1], s_v[c + 1], u1);
      u2 = fma(row[c + 2], s_v[c + 2], u2);
    }
    num = s_v[tid] * (u0 + u1 + u2);
    den = s_v[tid] * s_v[tid];
  }
  num = warp_sum(num);
  den = warp_sum(den);
  if (lane == 0) {
    s_red[warp][0] = num;
    s_red[warp][1] = den;
  }
  __syncthreads();
  if (tid == 0) {
    const double nn = s_red[0][0] + s_red[1][0], dd = s_red[0][1] + s_red[1][1];
    const double q = dd > 0.0 ? nn / dd : 0.0;
    lam[k] = isfinite(q) ? q : double(V[D * D + k]);  // else the float32 multisection value
    __threadfence();
    s_last = atomicAdd(done, 1u) == unsigned(D - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double l = tid < D ? __ldcg(&lam[tid]) : 0.0;
  double top = tid < D ? l : -1.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) top = fmax(top, __shfl_xor_sync(0xffffffffu, top, o));
  if (lane == 0) s_top[warp] = top;
  if (tid == 0) s_m = D - 1;  // m = D - 1 always passes
  __syncthreads();
  top = fmax(s_top[0], s_top[1]);
  if (tid < D && fabs(l) < kZeroEigRel * fmax(top, 1.0)) l = 0.0;
  if (tid < D) s_key[tid] = order_key(l);
  __syncthreads();
  if (tid < D) {
    const long long mine = s_key[tid];
    int rank = 0;
    for (int j = 0; j < D; ++j) {
      const long long o = s_key[j];
      rank += (o > mine) || (o == mine && j < tid);
    }
    s_sorted[rank] = l;
  }
  __syncthreads();
  if (tid == 0) {
    double acc = 0.0;
    for (int j = D - 1; j >= 0; --j) {
      acc += s_sorted[j];
      s_suffix[j] = acc;
    }
  }
  __syncthreads();
  if (tid < D) {
    const int cnt = D - tid;
    const double med = (cnt & 1) ? s_sorted[tid + cnt / 2]
                                 : 0.5 * (s_sorted[tid + cnt / 2 - 1] + s_sorted[tid + cnt / 2]);
    if (s_suffix[tid] <= med * double(cnt)) atomicMin(&s_m, tid);
    sc->eig[tid] = s_sorted[tid];
  }
  __syncthreads();
  if (tid == 0) {
    const int m = s_m;
    const double tau = s_suffix[m] / double(D - m);
    const double sg = sqrt(fmax(tau, 0.0));
    sc->m = m;
    sc->tau = tau;
    sc->sigma_est = sg;
    sc->ne_valid = 1;
    if (sigma_out) *sigma_out = sg;
    *done = 0u;  // ready for the next estimate
    __threadfence();
    atomicExch(&sc->sigma_ready, 1u);
  }
}

template <int W>
cudaError_t launch_wide(int stage, int n, int bits, int dtype, const GraphBufs& gb, const uint32_t* y8,
                        const float4* yf, float* spread, const WideNe& w, DevScalars* sc, double* sigma_out,
                        int num_sms, cudaStream_t stream) {
  constexpr int D = patch_dim<W>();
  const int P = D * D + D + 1;
  const int blocks = std::min(ne_wide_blocks(n, num_sms), w.blocks);
  switch (stage) {
    case 0:
      if (n <= 0) return cudaSuccess;
      if (dtype == 0) {
        static std::atomic<unsigned long long> configured{0};  // the shared-memory limit, once per device
        const cudaError_t e = once_per_device(configured, [] {
          return cudaFuncSetAttribute(k_ne_moments_wide_tc<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      int(WideGram<W>::SmemBytes));
        });
        if (e != cudaSuccess) return e;
        return launch_kernel(k_ne_moments_wide_tc<W>, dim3(blocks), dim3(kWThreads), WideGram<W>::SmemBytes, stream,
                             false, n, bits, gb, y8, spread, w.part);
      }
      return launch_kernel(k_ne_moments_wide_f32<W>, dim3(blocks), dim3(kWThreads), 0, stream, false, n, bits, gb,
                           yf, spread, w.part);
    case 1: {
      const int used = n > 0 ? blocks : 0;
      const dim3 rgrid((P + 31) / 32), rblock(32 * kReduceWarps);
      return dtype == 0 ? launch_kernel(k_ne_wide_reduce<0>, rgrid, rblock, 0, stream, false,
                                        static_cast<const double*>(w.part), used, D, w.tot)
                        : launch_kernel(k_ne_wide_reduce<1>, rgrid, rblock, 0, stream, false,
                                        static_cast<const double*>(w.part), used, D, w.tot);
    }
    case 2: {
      static std::atomic<unsigned long long> configured{0};  // the shared-memory limit, once per device
      const cudaError_t e = once_per_device(configured, [] {
        return cudaFuncSetAttribute(k_ne_wide_eigvec<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    int(wide_eig_smem<D>()));
      });
      if (e != cudaSuccess) return e;
      return launch_kernel(k_ne_wide_eigvec<D>, dim3(1), dim3(kWEigThreads), wide_eig_smem<D>(), stream, false,
                           static_cast<const double*>(w.tot), w.S, w.V, sc, sigma_out);
    }
    case 3:
      return launch_kernel(k_ne_wide_tail<D>, dim3(D), dim3(kWTailThreads), 0, stream, false,
                           static_cast<const double*>(w.tot), static_cast<const double*>(w.S),
                           static_cast<const float*>(w.V), w.lam, w.done, sc, sigma_out);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace

int ne_wide_blocks(int n, int num_sms) { return std::max(1, std::min((n + 127) / 128, 2 * num_sms)); }

size_t ne_wide_part_entries(int window) {
  const size_t D = size_t(3 * (6 * window + 1));
  return D * D + D + 1;
}

cudaError_t launch_ne_wide(int stage, int n, int bits, int window, int dtype, const GraphBufs& gb,
                           const uint32_t* y8, const float4* yf, float* spread, const WideNe& w, DevScalars* sc,
                           double* sigma_out, int num_sms, cudaStream_t stream) {
  if (gb.nx != extra_slots(window) || !w.part || !w.tot || !w.S || !w.V || !w.lam || !w.done)
    return cudaErrorInvalidValue;
  if (window == 2)
    return launch_wide<2>(stage, n, bits, dtype, gb, y8, yf, spread, w, sc, sigma_out, num_sms, stream);
  if (window == 3)
    return launch_wide<3>(stage, n, bits, dtype, gb, y8, yf, spread, w, sc, sigma_out, num_sms, stream);
  return cudaErrorInvalidValue;
}

}  // namespace fgbd
