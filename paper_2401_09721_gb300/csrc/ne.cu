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
constexpr int kSplits = 8;  // each tile's patch range split over 8 threads

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

struct NbKey {
  unsigned long long key;  // d^2, dz, dy, dx packed so that integer order is lexicographic
  int idx;                 // sorted id of the neighbour (input order among repeated voxels)
  float r, g, b;           // its colour, carried through the sort
};

__device__ __forceinline__ void cswap(NbKey& a, NbKey& b) {
  const bool sw = (b.key < a.key) || (b.key == a.key && b.idx < a.idx);
  if (sw) {
    const NbKey t = a;
    a = b;
    b = t;
  }
}

template <int DT>
__global__ void __launch_bounds__(kNeThreads)
    k_ne_moments(int n, int bits, const uint32_t* __restrict__ pk, const int4* __restrict__ c4,
                 const uint32_t* __restrict__ y8, const float4* __restrict__ yf,
                 float* __restrict__ spread, double* __restrict__ f64_partials, int moments,
                 DevScalars* __restrict__ sc) {
  // patches of one batch, transposed: row r holds entry r of the 256 patches
  __shared__ __align__(16) int8_t s_at8[DT == 0 ? kD : 1][kNeThreads];
  __shared__ __align__(16) float s_atf[DT == 1 ? kD : 1][kNeThreads];
  __shared__ unsigned long long s_red[kNeThreads / 32];

  const int tid = threadIdx.x;
  const int tile = tid / kSplits, split = tid % kSplits;
  int r0 = 0, c0 = 0;
  if (tid < kTiles * kSplits) tile_rc(tile, r0, c0);
  long long acc64[3][3] = {};
  double accd[3][3] = {};
  long long s1_64 = 0;
  double s1_d = 0.0;
  unsigned long long npatch = 0;

  for (int base = blockIdx.x * kNeThreads; base < n; base += gridDim.x * kNeThreads) {
    const int k = base + tid;
    bool has_patch = false;
    if (k < n) {
      const uint32_t ck = pk[k];
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

      float cr[7], cg[7], cb[7];
      if (DT == 0) {
        const uint32_t yk = y8[k];
        cr[6] = float(yk & 255u);
        cg[6] = float((yk >> 8) & 255u);
        cb[6] = float((yk >> 16) & 255u);
      } else {
        const float4 yk = yf[k];
        cr[6] = yk.x;
        cg[6] = yk.y;
        cb[6] = yk.z;
      }
      // gather neighbour colours (invalid slots repeat the point itself and are skipped below)
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        const int q = v[j] ? nb[j] : k;
        if (DT == 0) {
          const uint32_t yq = y8[q];
          cr[j] = float(yq & 255u);
          cg[j] = float((yq >> 8) & 255u);
          cb[j] = float((yq >> 16) & 255u);
        } else {
          const float4 yq = yf[q];
          cr[j] = yq.x;
          cg[j] = yq.y;
          cb[j] = yq.z;
        }
      }

      // FSLR spread over {k} and its neighbours, population std per channel
      const float cnt = float(deg + 1);
      float sp;
      if (DT == 0) {
        int sr = int(cr[6]), sg = int(cg[6]), sb = int(cb[6]);
        int qr = sr * sr, qg = sg * sg, qb = sb * sb;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          if (v[j]) {
            const int a = int(cr[j]), b = int(cg[j]), c = int(cb[j]);
            sr += a;
            sg += b;
            sb += c;
            qr += a * a;
            qg += b * b;
            qb += c * c;
          }
        }
        const int nn = deg + 1;
        const float vr = float(nn * qr - sr * sr), vg = float(nn * qg - sg * sg), vb = float(nn * qb - sb * sb);
        sp = (sqrtf(vr) / cnt + sqrtf(vg) / cnt + sqrtf(vb) / cnt) / 3.0f;
      } else {
        float mr = cr[6], mg = cg[6], mb = cb[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          if (v[j]) {
            mr += cr[j];
            mg += cg[j];
            mb += cb[j];
          }
        }
        mr /= cnt;
        mg /= cnt;
        mb /= cnt;
        float vr = (cr[6] - mr) * (cr[6] - mr), vg = (cg[6] - mg) * (cg[6] - mg), vb = (cb[6] - mb) * (cb[6] - mb);
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          if (v[j]) {
            vr += (cr[j] - mr) * (cr[j] - mr);
            vg += (cg[j] - mg) * (cg[j] - mg);
            vb += (cb[j] - mb) * (cb[j] - mb);
          }
        }
        sp = (sqrtf(vr / cnt) + sqrtf(vg / cnt) + sqrtf(vb / cnt)) / 3.0f;
      }
      spread[k] = sp;

      if (moments && deg == 6) {
        has_patch = true;
        // order the six neighbours by (d^2, dz, dy, dx, index)
        int kx, ky, kz;
        decode_c1(ck, bits, kx, ky, kz);
        NbKey e[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) {
          int x, y, z;
          decode_c1(pk[nb[j]], bits, x, y, z);
          const int dx = x - kx, dy = y - ky, dz = z - kz;
          const unsigned long long d2 = (unsigned long long)(dx * dx + dy * dy + dz * dz);
          e[j].key = (d2 << 33) | ((unsigned long long)(dz + 1024) << 22) |
                     ((unsigned long long)(dy + 1024) << 11) | (unsigned long long)(dx + 1024);
          e[j].idx = nb[j];
          e[j].r = cr[j];
          e[j].g = cg[j];
          e[j].b = cb[j];
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
        // write the patch, centred on 128, transposed into shared memory
        if (DT == 0) {
          s_at8[0][tid] = int8_t(int(cr[6]) - 128);
          s_at8[1][tid] = int8_t(int(cg[6]) - 128);
          s_at8[2][tid] = int8_t(int(cb[6]) - 128);
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            s_at8[3 + 3 * j][tid] = int8_t(int(e[j].r) - 128);
            s_at8[4 + 3 * j][tid] = int8_t(int(e[j].g) - 128);
            s_at8[5 + 3 * j][tid] = int8_t(int(e[j].b) - 128);
          }
        } else {
          s_atf[0][tid] = cr[6] - 128.f;
          s_atf[1][tid] = cg[6] - 128.f;
          s_atf[2][tid] = cb[6] - 128.f;
#pragma unroll
          for (int j = 0; j < 6; ++j) {
            s_atf[3 + 3 * j][tid] = e[j].r - 128.f;
            s_atf[4 + 3 * j][tid] = e[j].g - 128.f;
            s_atf[5 + 3 * j][tid] = e[j].b - 128.f;
          }
        }
      }
    }
    if (!moments) continue;
    if (!has_patch) {
#pragma unroll
      for (int r = 0; r < kD; ++r) {
        if (DT == 0) s_at8[r][tid] = 0;
        else s_atf[r][tid] = 0.f;
      }
    }
    npatch += has_patch ? 1 : 0;
    __syncthreads();

    if (tid < kTiles * kSplits) {
      if (DT == 0) {
        const int* at = reinterpret_cast<const int*>(&s_at8[0][0]);
        constexpr int kWordsPerRow = kNeThreads / 4;
        int acc[3][3] = {};
#pragma unroll
        for (int w = split * (kWordsPerRow / kSplits); w < (split + 1) * (kWordsPerRow / kSplits); ++w) {
          int a[3], b[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            a[i] = at[(r0 + i) * kWordsPerRow + w];
            b[i] = at[(c0 + i) * kWordsPerRow + w];
          }
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) acc[i][j] = __dp4a(a[i], b[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) acc64[i][j] += acc[i][j];
      } else {
        float acc[3][3] = {};
        constexpr int kPer = kNeThreads / kSplits;
#pragma unroll 4
        for (int p = split * kPer; p < (split + 1) * kPer; ++p) {
          float a[3], b[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            a[i] = s_atf[r0 + i][p];
            b[i] = s_atf[c0 + i][p];
          }
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) accd[i][j] += double(acc[i][j]);
      }
    } else if (tid < kTiles * kSplits + kD) {
      const int r = tid - kTiles * kSplits;
      if (DT == 0) {
        const int* at = reinterpret_cast<const int*>(&s_at8[0][0]);
        int acc = 0;
        for (int w = 0; w < kNeThreads / 4; ++w) acc = __dp4a(at[r * (kNeThreads / 4) + w], 0x01010101, acc);
        s1_64 += acc;
      } else {
        float acc = 0.f;
        for (int p = 0; p < kNeThreads; ++p) acc += s_atf[r][p];
        s1_d += double(acc);
      }
    }
    __syncthreads();
  }
  if (!moments) return;

  // combine the 8 splits of each tile (8 consecutive lanes)
  const unsigned long long np = block_sum_u64<kNeThreads>(npatch, s_red);
  if (tid == 0 && DT == 0 && np) atomicAdd(&sc->n_patches, np);
  if (tid < kTiles * kSplits) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        long long v64 = acc64[i][j];
        double vd = accd[i][j];
#pragma unroll
        for (int o = 1; o < kSplits; o <<= 1) {
          v64 += __shfl_xor_sync(0xffffffffu, v64, o);
          vd += __shfl_xor_sync(0xffffffffu, vd, o);
        }
        acc64[i][j] = v64;
        accd[i][j] = vd;
      }
    if (split == 0) {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int idx = (r0 + i) * kD + (c0 + j);
          if (DT == 0) {
            if (acc64[i][j]) atomicAdd(reinterpret_cast<unsigned long long*>(&sc->s2[idx]),
                                       (unsigned long long)acc64[i][j]);
          } else {
            f64_partials[size_t(blockIdx.x) * (kD * kD + kD + 1) + idx] = accd[i][j];
          }
        }
    }
  } else if (tid < kTiles * kSplits + kD) {
    const int r = tid - kTiles * kSplits;
    if (DT == 0) {
      if (s1_64) atomicAdd(reinterpret_cast<unsigned long long*>(&sc->s1[r]), (unsigned long long)s1_64);
    } else {
      f64_partials[size_t(blockIdx.x) * (kD * kD + kD + 1) + kD * kD + r] = s1_d;
    }
  }
  if (DT == 1 && tid == 0)
    f64_partials[size_t(blockIdx.x) * (kD * kD + kD + 1) + kD * kD + kD] = double(np);
}

// ---------------------------------------------------------------- finalize

constexpr double kZeroEigRel = 1e-10;  // relative size below which an eigenvalue is zero
constexpr int kJ = 22;           // 21 padded to an even size for round-robin pairing
constexpr int kMaxSweeps = 12;

__global__ void __launch_bounds__(256) k_ne_finalize(int dtype, const double* __restrict__ f64_partials,
                                                     int nblocks, DevScalars* __restrict__ sc,
                                                     double* __restrict__ sigma_out) {
  __shared__ double S[kD][kD];
  __shared__ double s_sum[kD * kD + kD + 1];
  __shared__ float A[kJ][kJ + 1];
  __shared__ float V[kJ][kJ + 1];
  __shared__ float s_c[kJ / 2], s_s[kJ / 2];
  __shared__ int s_p[kJ / 2], s_q[kJ / 2];
  __shared__ double s_lam[kD];
  __shared__ double s_sorted[kD];
  __shared__ double s_num[kD][kD];

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
  for (int e = tid; e < kD * kD; e += blockDim.x) {
    const int r = e / kD, c = e % kD;
    const int rr = min(r, c), cc = max(r, c);
    const double mr = s_sum[kD * kD + rr] / npd, mc = s_sum[kD * kD + cc] / npd;
    S[r][c] = s_sum[rr * kD + cc] / npd - mr * mc;
  }
  __syncthreads();
  for (int e = tid; e < kJ * kJ; e += blockDim.x) {
    const int r = e / kJ, c = e % kJ;
    A[r][c] = (r < kD && c < kD) ? float(S[r][c]) : 0.f;
    V[r][c] = (r == c) ? 1.f : 0.f;
  }
  __syncthreads();

  // cyclic Jacobi, round-robin order: 11 disjoint rotations per round.  A pair
  // is rotated only while |a_pq| >= 1e-7 sqrt|a_pp a_qq| (float32 resolution);
  // a sweep that rotates nothing ends the iteration.
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    int rotated = 0;
    for (int round = 0; round < kJ - 1; ++round) {
      int did = 0;
      if (tid < kJ / 2) {
        int p, q;
        if (tid == 0) {
          p = round;
          q = kJ - 1;
        } else {
          p = (round + tid) % (kJ - 1);
          q = (round - tid + (kJ - 1)) % (kJ - 1);
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        const float apq = A[p][q], app = A[p][p], aqq = A[q][q];
        float c = 1.f, s = 0.f;
        if (fabsf(apq) >= 1e-7f * sqrtf(fabsf(app * aqq)) && apq != 0.f) {
          const float theta = (aqq - app) / (2.f * apq);
          const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
          c = rsqrtf(t * t + 1.f);
          s = t * c;
          did = 1;
        }
        s_p[tid] = p;
        s_q[tid] = q;
        s_c[tid] = c;
        s_s[tid] = s;
      }
      const int any = __syncthreads_count(did);
      rotated += any;
      if (!any) continue;
      // rows: A <- J^T A
      for (int e = tid; e < (kJ / 2) * kJ; e += blockDim.x) {
        const int pr = e / kJ, j = e % kJ;
        const int p = s_p[pr], q = s_q[pr];
        const float c = s_c[pr], s = s_s[pr];
        const float ap = A[p][j], aq = A[q][j];
        A[p][j] = c * ap - s * aq;
        A[q][j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = tid; e < (kJ / 2) * kJ; e += blockDim.x) {
        const int pr = e / kJ, i = e % kJ;
        const int p = s_p[pr], q = s_q[pr];
        const float c = s_c[pr], s = s_s[pr];
        const float ap = A[i][p], aq = A[i][q];
        A[i][p] = c * ap - s * aq;
        A[i][q] = s * ap + c * aq;
        const float vp = V[i][p], vq = V[i][q];
        V[i][p] = c * vp - s * vq;
        V[i][q] = s * vp + c * vq;
      }
      __syncthreads();
    }
    if (rotated == 0) break;
  }

  // float64 Rayleigh quotients of the 21 eigenvector estimates
  for (int e = tid; e < kD * kD; e += blockDim.x) {
    const int k = e / kD, r = e % kD;
    double w = 0.0;
    for (int c = 0; c < kD; ++c) w += S[r][c] * double(V[c][k]);
    s_num[k][r] = w * double(V[r][k]);
  }
  __syncthreads();
  if (tid < kD) {
    double num = 0.0, den = 0.0;
    for (int r = 0; r < kD; ++r) {
      num += s_num[tid][r];
      den += double(V[r][tid]) * double(V[r][tid]);
    }
    s_lam[tid] = num / den;
  }
  __syncthreads();
  // eigenvalues below 1e-10 max(lambda_1, 1) are numerical zeros (a rank-deficient
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
  if (tid == 0) {
    // tail rule: smallest m with mean(lambda_{m+1..D}) <= median(lambda_{m+1..D})
    double suffix[kD + 1];
    suffix[kD] = 0.0;
    for (int i = kD - 1; i >= 0; --i) suffix[i] = suffix[i + 1] + s_sorted[i];
    int m = kD - 1;
    double tau = s_sorted[kD - 1];
    for (int mm = 0; mm < kD; ++mm) {
      const int cnt = kD - mm;
      const double mean = suffix[mm] / double(cnt);
      const double med = (cnt & 1) ? s_sorted[mm + cnt / 2]
                                   : 0.5 * (s_sorted[mm + cnt / 2 - 1] + s_sorted[mm + cnt / 2]);
      if (mean <= med) {
        m = mm;
        tau = mean;
        break;
      }
    }
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
  return std::max(1, std::min((n + kNeThreads - 1) / kNeThreads, num_sms * 4));
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
  k_ne_finalize<<<1, 256, 0, stream>>>(dtype, f64_partials, nblocks, sc, sigma_out);
  return cudaGetLastError();
}

}  // namespace fgbd
