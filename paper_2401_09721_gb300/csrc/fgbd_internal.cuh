// Internal declarations shared by the FGBD CUDA translation units.
//
// Index spaces.  The caller's points are in "input order".  Internally every
// per-point array is kept in "sorted order": the order of the first scan-line
// code C1 = 2^{2b} z + 2^b y + x (Section 2.2, Eq. 1).  In that order the two
// code-1 neighbours of point k are simply k-1 and k+1, and the packed C1 code
// of point k doubles as its coordinates.  Neighbours along C2 and C3
// (Eq. 2-3) are stored explicitly, four slots per point, with -1 marking an
// empty slot (the end of a scan order, or a pair already linked by an earlier
// code, so that the union graph of Section 2.2 is a set).  With a window
// w > 1 the points d = 2..w positions away along each code are stored in
// 6 (w - 1) further slots per point (GraphBufs::cx).
#pragma once

#include <atomic>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace fgbd {

constexpr int kMaxBits = 10;                       // three b-bit coordinates fit a 32-bit code
constexpr int kMaxRadix = 1 << kMaxBits;           // radix passes use one coordinate (b bits) as digit
constexpr int kSortThreads = 256;
constexpr int kSortKpt = 16;                       // keys per thread
constexpr int kSortTile = kSortThreads * kSortKpt;  // 4096 keys per tile
constexpr int kSlgPasses = 3;                      // y-slabs (then the slab sort: C3), C1, C2
constexpr int kK = 6;                              // neighbours per point at window 1
constexpr int kD = 3 * (kK + 1);                   // patch dimension (Section 2.3)
constexpr int kMaxWindow = 3;                      // windows 1..3: K = 6w neighbours per point
constexpr int kDMax = 3 * (6 * kMaxWindow + 1);    // largest patch dimension (57)
constexpr int kQCap = 256;                         // largest q_max accepted
constexpr int kSqShift = 8;                        // fixed point of squared colours (2^-8)
constexpr int kDistShift = 20;                     // fixed point of edge lengths
constexpr int kNeThreads = 256;
constexpr int kFilterThreads = 512;
constexpr int kSpecMax = 3;                        // filter steps taken while sigma_est is computed
constexpr uint32_t kCoordMask = 0x3FFFFFFFu;       // low 30 bits: packed C1 code
// The two high bits of a sorted point's packed code (pk, and x.w of an iterate)
// mark a missing link to its C1 neighbour k - 1 / k + 1: set by the link step
// only under the same-line variant, zero otherwise.
constexpr uint32_t kNoPrevLink = 1u << 30;
constexpr uint32_t kNoNextLink = 1u << 31;
constexpr uint32_t kKeepBit = 0x80000000u;         // FSLR keep flag beside the code

// latched device error bits
enum : uint32_t {
  kFlagRange = 1u,    // a coordinate outside [0, 2^b)
  kFlagTimeout = 2u,  // a bounded device-side wait gave up
};

// Device-resident scalars of one context.  Regions are zeroed separately by
// the call that fills them (see the offsets used in api.cu).
struct DevScalars {
  // ---- graph build region
  unsigned long long n_edges;   // distinct undirected edges E
  unsigned long long dist_fx;   // sum of edge lengths, fixed point 2^-kDistShift
  alignas(16) uint32_t chist[3][kMaxRadix];  // histograms of x, y and z (read as uint4)
  unsigned long long node_fx;   // node-mean reading: sum over points of their mean edge length (fixed point)
  unsigned long long node_cnt;  // and the points that have edges
  float cexp;                   // the Eq. 4 exponent scale log2(e) / sigma_g^2 of this graph, once cexp_ready
  uint32_t cexp_ready;          // set by the first moments launch on this graph
  uint32_t build_end_;
  // ---- noise estimate region
  unsigned long long n_patches;
  long long s1[kD];             // sum of (a - 128)
  long long s2[kD * kD];        // sum of (a - 128)(a - 128)^T (upper triangle filled)
  uint32_t spec_barrier;        // grid barrier of the speculative filter steps
  int32_t spec_done;            // filter steps stored by the noise-estimate kernel
  uint32_t sigma_ready;         // set (release) once sigma_est of this estimate is written
  uint32_t spec_go[kSpecMax + 1];  // after stored step t: 1 to take another before selecting
  float fslr_thr[4];            // the FSLR threshold of this sigma_est as the selection uses it (once fslr_ready)
  uint32_t fslr_ready;          // set by the eigen step with sigma_est
  uint32_t ne_end_;
  // ---- results of the noise estimate
  double eig[kDMax];            // descending (the first D = 3 (6w + 1) are used)
  double tau;
  double sigma_est;
  int32_t m;
  int32_t ne_valid;
  // ---- selection region
  unsigned long long ysq_keep;  // fixed point 2^-kSqShift
  unsigned long long ysq_all;
  unsigned long long n_keep;
  unsigned long long sumsq[kQCap + 1];
  long long spec_keep[kSpecMax + 1];  // over the kept points: sum of x_q^2 (fixed point), stored steps q = 1..
  long long spec_all[kSpecMax + 1];   // the same over every point
  uint32_t barrier;
  uint32_t sel_end_;
  // ---- results of the selection
  double J[kQCap + 1];
  int32_t kept_buf;             // where x_q is: 0 / 1 the iterate buffers, 2 + q - 1 a stored step, -1 the input,
                                // kKeptBest the copy of the global reading's best iterate
  int32_t q_sel;
  int32_t n_J;
  int32_t sel_valid;
  // ---- latched errors (never zeroed by a call; cleared when read)
  uint32_t status;
  // ---- settings (set at context creation)
  unsigned long long wait_limit_ns;  // any device-side wait gives up after this long
  uint32_t sigma_mode;               // sigma_g of Eq. 4: kSigmaEdge, kSigmaNode or kSigmaPair
  uint32_t pooled_patch;             // 1: patches of D = 7 pooled over the colour channels (Section 2.3)
  double fslr_factor;                // the FSLR threshold factor (2 in Section 2.4)
};

// Readings of sigma_g (Section 2.2): the mean length over the edges (the
// method as read here), the mean over the points of each point's mean edge
// length, or a bandwidth per point (w_ij = exp(-d_ij^2 / (sigma_i sigma_j))).
enum : uint32_t { kSigmaEdge = 0u, kSigmaNode = 1u, kSigmaPair = 2u };

// the regions are zeroed as 32-bit words
static_assert(offsetof(DevScalars, n_edges) % 4 == 0 && offsetof(DevScalars, build_end_) % 4 == 0 &&
                  offsetof(DevScalars, n_patches) % 4 == 0 && offsetof(DevScalars, ne_end_) % 4 == 0 &&
                  offsetof(DevScalars, ysq_keep) % 4 == 0 && offsetof(DevScalars, sel_end_) % 4 == 0,
              "DevScalars regions must be whole 32-bit words");
static_assert(offsetof(DevScalars, n_edges) < offsetof(DevScalars, build_end_) &&
                  offsetof(DevScalars, build_end_) < offsetof(DevScalars, n_patches) &&
                  offsetof(DevScalars, ne_end_) < offsetof(DevScalars, ysq_keep),
              "the build, noise and selection regions are zeroed as one range by fgbd_run");

// Sort scratch for one build.
struct SortBufs {
  uint32_t* keys[2];     // ping-pong [cap]
  uint32_t* vals[2];     // ping-pong [cap]
  uint32_t* tile_counts; // [3 passes][kMaxRadix digits][tiles of the capacity]: per-tile digit counts,
                         // then offsets.  Pass 0's are written by the histogram launch, pass 1's
                         // added up by the slab sort (zeroed by the histogram launch), pass 2's by
                         // a counting launch.
  int count_stride;      // words of one pass's counts: kMaxRadix * tiles of the capacity
};

// Graph in sorted order.
struct GraphBufs {
  int32_t* perm1;    // [cap] input index of each sorted (C1-order) point
  int32_t* rank1;    // [cap] sorted id of each input point
  uint32_t* pk;      // [cap] packed C1 code of each sorted point (its coordinates)
  int32_t* ord23;    // [2][cap] sorted ids along C2, then along C3
  int32_t* rank2;    // [cap] position of each sorted id in the C2 order
  int4* c4;          // [cap] C2 prev, C2 next, C3 prev, C3 next (sorted ids, -1 empty)
  // windows w > 1: [6 (w - 1)][cap stride] the points d = 2..w positions away;
  // slot 6 (d - 2) + 2 l + s holds code l's point d before (s = 0) / after (s = 1)
  // the point (sorted ids, -1 empty or linked by an earlier code)
  int32_t* cx;
  int nx;            // 6 (w - 1)
  int cx_stride;     // row stride of cx, a multiple of 64
  float* node_sig;   // [cap] each sorted point's mean edge length (the node and pair readings of sigma_g), or null
};

// number of further neighbour slots at window w
__host__ __device__ constexpr int extra_slots(int w) { return 6 * (w - 1); }

// One stable radix pass whose digit is one coordinate field of the key.
struct SortPassArgs {
  int n;
  int bits;
  int tiles;
  int shift;               // bit offset of the digit in the key
  int coord;               // which coordinate histogram gives the digit totals
  const int32_t* xyz;      // if set: keys from the coordinates, values = input index
  const uint32_t* keys_in;
  const uint32_t* vals_in; // null: value = position
  uint32_t* keys_out;      // null: not written
  uint32_t* vals_out;
  int32_t* rank_out;       // rank_out[value] = output position, or null
  int32_t* pos_out;        // pos_out[input position] = output position, or null
  int pass;                // 0, 1, 2 (which launch made the tile counts: pass_counted_before)
  uint32_t* counts;
  const DevScalars* sc;
};

// ---------------------------------------------------------------- segmented launches
// A batch of frames runs each stage as one launch: the per-frame arguments of
// up to kSegMax frames travel in the kernel's parameter space, and frame f
// owns the blocks [start[f], start[f + 1]) of a one-dimensional grid.  A
// block finds its frame, then runs the same body as the one-frame kernel with
// its block index and block count inside the frame, so a frame's results do
// not depend on the batch it is in.
constexpr int kSegMax = 16;

template <typename A>
struct Seg {
  A a[kSegMax];
  int start[kSegMax + 1];
  int count;
};

// the frame that owns block b (frames with no blocks are skipped)
template <typename A>
__device__ __forceinline__ int seg_frame(const Seg<A>& s, int b) {
  int f = 0;
  while (f + 1 < s.count && s.start[f + 1] <= b) ++f;
  return f;
}

// fill s.start from per-frame block counts; returns the grid size
template <typename A>
inline int seg_layout(Seg<A>& s, const int* blocks, int count) {
  s.count = count;
  int t = 0;
  for (int f = 0; f < count; ++f) {
    s.start[f] = t;
    t += blocks[f];
  }
  s.start[count] = t;
  return t;
}

// Arguments of the kernels that the one-frame path passes one by one.
struct HistArgs {
  const int32_t* xyz;
  int n;
  int bits;
  struct DevScalars* sc;
  uint32_t* counts0;     // sort pass 0's tile counts (the y digits of each 4096-point input tile), or null
  uint32_t* counts1;     // pass 1's tile counts, zeroed here (the slab sort adds them up), or null
};
struct SlabArgs {
  int n;
  int bits;
  const uint32_t* keys_in;
  const uint32_t* vals_in;
  uint32_t* keys_tmp;
  uint32_t* vals_tmp;
  uint32_t* keys_out;
  int32_t* vals_out;
  const struct DevScalars* sc;
  uint32_t* counts1;     // sort pass 1's tile counts: the z digits of the C3 order, added up here (or null)
};
struct LinkArgs {
  int n;
  int bits;
  int cap;
  const int32_t* ord23;
  const uint32_t* keys_c2;
  const uint32_t* keys_c3;
  const int32_t* rank2;
  uint32_t* pk;
  int4* c4;
  struct DevScalars* sc;
};
struct GatherArgs {
  const void* rgb;
  int dtype;
  int n;
  const int32_t* perm1;
  uint32_t* y8;
  float4* yf;
};
struct MomentArgs {
  int n;
  int bits;
  const uint32_t* pk;
  const int4* c4;
  const uint32_t* y8;
  const float4* yf;
  float* spread;
  double* f64_partials;
  int moments;
  int sorted_patches;
  struct DevScalars* sc;
  float4* x0;  // if set: also x_0 of the filter steps, (r, g, b, packed code) per sorted point
};
struct ZeroArgs {
  uint32_t* p;
  size_t words;
};

// How a batch runs, chosen by the batch tuner (api.cu): frames per segmented
// launch (0: every frame on a stream of its own, its own kernels), threads of
// the sort scatter (one 4096-key tile a block), threads of the filter blocks
// and filter blocks per SM of the cooperative selection.
struct BatchShape {
  int seg_frames = kSegMax;
  int scatter_threads = 512;
  int filter_threads = 512;
  int filter_per_sm = 2;
};

// ---------------------------------------------------------------- launchers
struct FilterArgs;
// Every launcher enqueues on `stream` and returns the launch error.

// the coordinate histograms; with sb, also sort pass 0's tile counts (and pass 1's zeroed)
cudaError_t launch_coord_hist(const int32_t* xyz, int n, int bits, DevScalars* sc, const SortBufs* sb, int num_sms,
                              cudaStream_t stream);
// pass 0: y-slabs from the input; (the slab sort then gives C3); pass 1: C1 = the C3 order on z;
// pass 2: C2 = the C1 order on x
SortPassArgs slg_pass_args(int pass, const int32_t* xyz, int n, int bits, int cap, const SortBufs& sb,
                           const GraphBufs& gb, const DevScalars* sc);
// C3 within each y-slab (after pass 0): (x, z) order into keys[1] and ord23[1]
cudaError_t launch_slab_sort(int n, int bits, int cap, const SortBufs& sb, const GraphBufs& gb,
                             const DevScalars* sc, cudaStream_t stream);
cudaError_t launch_tile_counts(const SortPassArgs& a, cudaStream_t stream);
// pass p's tile counts are made by the launches before it for p = 0 (histogram) and p = 1 (slab sort)
constexpr bool pass_counted_before(int pass) { return pass < 2; }
cudaError_t launch_tile_scan(const SortPassArgs& a, cudaStream_t stream);
cudaError_t launch_sort_scatter(const SortPassArgs& a, cudaStream_t stream);
cudaError_t launch_sort_pass(const SortPassArgs& a, cudaStream_t stream);  // the three above
cudaError_t launch_orders_export(int n, int cap, const GraphBufs& gb, int32_t* out, cudaStream_t stream);
// segmented launches: one launch for frames 0..count-1 (count <= kSegMax), each
// frame with the blocks its one-frame launch would have
HistArgs hist_args(const int32_t* xyz, int n, int bits, DevScalars* sc, const SortBufs& sb);
LinkArgs link_args(int n, int bits, int cap, const GraphBufs& gb, const SortBufs& sb, DevScalars* sc);
cudaError_t launch_zero_words_seg(const ZeroArgs* a, int count, cudaStream_t stream);
cudaError_t launch_coord_hist_seg(const HistArgs* a, int count, int num_sms, cudaStream_t stream);
// counts, scan and scatter of one pass (scatter_threads: 256, 512 or 1024 per 4096-key tile)
cudaError_t launch_sort_pass_seg(const SortPassArgs* a, int count, int scatter_threads, cudaStream_t stream);
cudaError_t launch_slab_sort_seg(const int* n, const int* bits, const int* cap, const SortBufs* sb,
                                 const GraphBufs* gb, DevScalars* const* sc, int count, cudaStream_t stream);
cudaError_t launch_link_seg(const LinkArgs* a, int count, bool same_line, int num_sms, cudaStream_t stream);
cudaError_t launch_link(int n, int bits, int cap, bool same_line, const GraphBufs& gb, const SortBufs& sb,
                        DevScalars* sc, int num_sms, cudaStream_t stream);
// each sorted point's mean edge length into gb.node_sig (if set) and, for the
// node reading of sigma_g, their sum and count into the build scalars
cudaError_t launch_node_sigma(int n, int bits, const GraphBufs& gb, DevScalars* sc, int num_sms, cudaStream_t stream);
// windows w > 1: every link of the window (C2/C3 d = 1 into c4, d >= 2 into cx)
// and the edge sums; then k_c1_line_flags under the same-line variant
cudaError_t launch_link_wide(int n, int bits, int cap, int window, bool same_line, const GraphBufs& gb,
                             const SortBufs& sb, DevScalars* sc, int num_sms, cudaStream_t stream);

cudaError_t launch_gather_colors(const void* rgb, int dtype, int n, const int32_t* perm1,
                                 uint32_t* y8, float4* yf, cudaStream_t stream);
// x0: if set, the launch also writes x_0 of the filter steps (colours and packed code)
cudaError_t launch_ne_moments(int n, int bits, int dtype, const GraphBufs& gb, const uint32_t* y8,
                              const float4* yf, float* spread, double* f64_partials,
                              DevScalars* sc, int num_sms, bool moments, bool sorted_patches,
                              cudaStream_t stream, float4* x0 = nullptr);
// spec: if not null (and spec->spec_depth > 0), the same launch also takes the
// first spec_depth filter steps on the other SMs (one block per SM)
cudaError_t launch_ne_finalize(int dtype, const double* f64_partials, int nblocks,
                               DevScalars* sc, double* sigma_out, const FilterArgs* spec, int num_sms,
                               cudaStream_t stream);
int ne_moment_blocks(int n, int num_sms);
// testing: div_newton and CUDA's division of n operand pairs
cudaError_t launch_debug_div(const double* a, const double* b, double* q_newton, double* q_div, int64_t n,
                             cudaStream_t stream);
MomentArgs moment_args(int n, int bits, const GraphBufs& gb, const uint32_t* y8, const float4* yf, float* spread,
                       double* f64_partials, bool moments, bool sorted_patches, DevScalars* sc);
// segmented: frames 0..count-1 (count <= kSegMax; one colour dtype for the moments)
cudaError_t launch_gather_colors_seg(const GatherArgs* a, int count, cudaStream_t stream);
cudaError_t launch_ne_moments_seg(const MomentArgs* a, int count, int dtype, int num_sms, cudaStream_t stream);
// the estimate launch over frames: one eigen block per frame, the other SMs
// shared out for the speculative steps (spec[f].spec_depth of them)
cudaError_t launch_ne_finalize_seg(const FilterArgs* spec, const double* const* f64_partials, const int* nblocks,
                                   int count, int num_sms, cudaStream_t stream);

// Noise estimate at windows w > 1 (patch dimension D = 3 (6w + 1)): per-block
// moment partials, their reduction, the one-block float32 eigenvectors, and float64
// Rayleigh quotients with the tail rule.
struct WideNe {
  double* part;   // [blocks][D*D + D + 1] per-block moments (int64 bit patterns for uint8 colours)
  double* tot;    // [D*D + D + 1] the totals: sum a a^T (upper triangle), sum a, patch count
  double* S;      // [D][D] the covariance
  float* V;       // [D][D] its eigenvector estimates (columns), then their D float32 eigenvalues
  double* lam;    // [D] Rayleigh quotients
  uint32_t* done; // blocks of the Rayleigh launch finished (reset by the last)
  int blocks;     // moment blocks (the rows of part)
};
int ne_wide_blocks(int n, int num_sms);
size_t ne_wide_part_entries(int window);  // D*D + D + 1
// stage 0 the moments (nothing at n = 0), 1 their reduction, 2 the eigenvector block, 3 the tail rule
cudaError_t launch_ne_wide(int stage, int n, int bits, int window, int dtype, const GraphBufs& gb,
                           const uint32_t* y8, const float4* yf, float* spread, const WideNe& w, DevScalars* sc,
                           double* sigma_out, int num_sms, cudaStream_t stream);

struct FilterArgs {
  int n;
  int bits;
  int dtype;             // colours held in y8 (0) or yf (1)
  int mode;              // 0: select q (Eq. 6), 1: fixed q
  int q_fixed;           // mode 1
  const int32_t* q_src;  // mode 1: if set, q is read here on the device (and q_sel is left as it is)
  int q_max;             // mode 0
  double fslr_factor;
  int all_points;        // Eq. 6 over every point (the limited region is off)
  const double* sigma_src;  // sigma_est to use (device)
  const uint32_t* y8;
  const float4* yf;
  const float* spread;
  const uint32_t* pk;
  const int4* c4;
  const int32_t* rank1;
  float4* xbuf0;
  float4* xbuf1;
  void* out;             // input-order output or nullptr
  int out_dtype;
  DevScalars* sc;
  // select mode: the first spec_depth steps were stored before sigma_est was known
  int spec_depth;          // 0: none
  const float4* x0;        // x_0 as the moments launch wrote it (r, g, b, packed code), or null: from y8/yf, pk
  float4* spec_x;          // [kSpecMax][cap]: x_1 .. x_S
  int32_t* spec_z;         // [kSpecMax][cap]: per point sum_c x_q^2, fixed point
  int cap;                 // row stride of spec_x / spec_z, a multiple of 64
  int fuse;                // noise-estimate launch: select and filter too, once sigma_est is known
  uint8_t* keep8;          // select mode: the FSLR keep flag of every sorted point
  // windows w > 1: the further neighbour slots (GraphBufs::cx), nx = 6 (w - 1)
  const int32_t* cx;
  int nx;
  int cx_stride;
  // the pair reading of sigma_g: each sorted point's mean edge length (null otherwise)
  const float* node_sig;
  // the global reading of the q search: argmin of J over 0..q_max; the best
  // iterate beyond the stored steps is copied to xbest
  int q_global;
  float4* xbest;
  // window 1: the Eq. 4 weights of each sorted point's six slots, normalised by
  // their sum (slots C1 prev, C1 next, C2 prev, C2 next in w4; C3 prev, next in
  // w2), written by step 1 and read by every later step of the same graph
  float4* w4;
  float2* w2;
};
constexpr int kKeptBest = 64;  // kept_buf value of the iterate copied to xbest
cudaError_t launch_filter(const FilterArgs& a, int grid, cudaStream_t stream);
int filter_grid(int n, int num_sms, int nx = 0);
cudaError_t launch_output(const FilterArgs& a, cudaStream_t stream);  // the kept iterate, in input order
// the cooperative selection/filter over frames (window 1): filter_per_sm blocks
// of `threads` (256 or 512) per SM, shared out in proportion to the frames' points
cudaError_t launch_filter_seg(const FilterArgs* a, int count, int threads, int filter_per_sm, int num_sms,
                              cudaStream_t stream);
int filter_seg_max_per_sm(int threads);  // resident blocks per SM of that kernel

// Differentiable filter: rows of R = D^-1 W for given alpha, sigma, and their transpose
struct DiffBufs {
  int32_t* nb;  // [n][6] neighbour ids (sorted order), -1 unused
  float* R;     // [n][6] R_ij
  float* RT;    // [n][6] R_ji: weight of i in the row of its t-th neighbour
  float* d2;    // [n][6] squared distances
  float* e;     // [n] sum_j R_ij d_ij^2
};
int diff_grid(int n, int num_sms);
cudaError_t launch_diff_rows(int n, int bits, double sigma, const GraphBufs& gb, const DevScalars* sc,
                             const DiffBufs& db, int num_sms, cudaStream_t stream);
cudaError_t launch_diff_gather(int n, const float* rgb, const int32_t* perm1, float4* x, int num_sms,
                               cudaStream_t stream);
cudaError_t launch_diff_scatter(int n, const float4* x, const int32_t* perm1, float* out, int num_sms,
                                cudaStream_t stream);
cudaError_t launch_diff_step(int n, float alpha, const DiffBufs& db, const float4* src, float4* dst, int num_sms,
                             cudaStream_t stream);
cudaError_t launch_diff_back_step(int n, float alpha, double sigma, const DiffBufs& db, const float4* x,
                                  const float4* u, float4* u_out, const DevScalars* sc, double* partial,
                                  int num_sms, cudaStream_t stream);
cudaError_t launch_diff_reduce(int count, const double* partial, double* grad, cudaStream_t stream);

// CSR export in input order
cudaError_t launch_csr_degree(int n, const GraphBufs& gb, int64_t* deg_out, cudaStream_t stream);
cudaError_t launch_scan_i64(int64_t* data, int64_t count, int64_t* block_tmp, cudaStream_t stream);
cudaError_t launch_csr_fill(int n, int bits, const GraphBufs& gb, const int64_t* row_ptr, int32_t* col,
                            float* w, int64_t col_capacity, const DevScalars* sc, cudaStream_t stream);
cudaError_t launch_spread_export(int n, const int32_t* rank1, const float* spread, const uint8_t* keep8,
                                 float* spread_out, uint8_t* keep_out, cudaStream_t stream);

// ---------------------------------------------------------------- device helpers

__host__ __device__ inline uint32_t code_of(int which, uint32_t x, uint32_t y, uint32_t z, int b) {
  // Eq. 1-3 with the three b-bit fields packed high to low
  switch (which) {
    case 0: return (z << (2 * b)) | (y << b) | x;
    case 1: return (x << (2 * b)) | (z << b) | y;
    default: return (y << (2 * b)) | (x << b) | z;
  }
}

// an index read from device memory is used only if it lies in [0, n)
__device__ __forceinline__ bool in_range(int v, int n) { return unsigned(v) < unsigned(n); }

__device__ __forceinline__ void decode_c1(uint32_t c, int b, int& x, int& y, int& z) {
  const uint32_t m = (1u << b) - 1u;
  x = int(c & m);
  y = int((c >> b) & m);
  z = int((c >> (2 * b)) & m);
}

// whether sorted point k is linked to k - 1 / k + 1 (C1 neighbours), from its packed-code word
__device__ __forceinline__ bool c1_prev_linked(uint32_t pkw, int k) { return k > 0 && !(pkw & kNoPrevLink); }
__device__ __forceinline__ bool c1_next_linked(uint32_t pkw, int k, int n) { return k + 1 < n && !(pkw & kNoNextLink); }

// Neighbour j (0 .. 5 + nx) of sorted point k in link order: 0 / 1 the C1
// points k - 1 / k + 1 (pkw: k's packed-code word with the missing-link
// bits), 2..5 the c4 slots s, then the further slots of a window w > 1.
// Returns its sorted id, or -1 for an empty slot.
__device__ __forceinline__ int neighbour_of(int j, int k, int n, uint32_t pkw, int4 s, const int32_t* __restrict__ cx,
                                            int cx_stride) {
  int v;
  switch (j) {
    case 0: return c1_prev_linked(pkw, k) ? k - 1 : -1;
    case 1: return c1_next_linked(pkw, k, n) ? k + 1 : -1;
    case 2: v = s.x; break;
    case 3: v = s.y; break;
    case 4: v = s.z; break;
    case 5: v = s.w; break;
    default: v = cx[size_t(j - 6) * size_t(cx_stride) + k]; break;
  }
  return in_range(v, n) ? v : -1;
}

__device__ __forceinline__ int sq_dist_c1(uint32_t a, uint32_t c, int b) {
  int ax, ay, az, cx, cy, cz;
  decode_c1(a, b, ax, ay, az);
  decode_c1(c, b, cx, cy, cz);
  const int dx = cx - ax, dy = cy - ay, dz = cz - az;
  return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s for any device-side wait

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}
__device__ __forceinline__ void st_volatile(uint32_t* p, uint32_t v) {
  *reinterpret_cast<volatile uint32_t*>(p) = v;
}

// round(v^2 * 2^kSqShift) as a 32-bit integer: exact for integer colours,
// within 2^-9 otherwise; colours on the 0..255 scale (|v| < 2896) fit.
// A 32-bit conversion keeps the per-point work off the float64 pipe.
__device__ __forceinline__ int sq_fixed(float v) { return __float2int_rn(v * v * float(1 << kSqShift)); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of a 64-bit counter, result valid in thread 0
template <int THREADS>
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v,
                                                            unsigned long long* smem) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) smem[warp] = v;
  __syncthreads();
  unsigned long long t = 0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < THREADS / 32; ++w) t += smem[w];
  }
  __syncthreads();
  return t;
}

// sigma_g (Section 2.2) from the build sums: the mean edge length, or under
// the node reading the mean of the points' mean edge lengths
__device__ __forceinline__ double sigma_g_of(const DevScalars* sc) {
  if (sc->sigma_mode == kSigmaNode) {
    const unsigned long long c = sc->node_cnt;
    return c ? double(sc->node_fx) * (1.0 / double(1ull << kDistShift)) / double(c) : 0.0;
  }
  const unsigned long long e = sc->n_edges;
  if (e == 0) return 0.0;
  return double(sc->dist_fx) * (1.0 / double(1ull << kDistShift)) / double(e);
}

// ---------------------------------------------------------------- launches
// Programmatic dependent launch (opt-in): with FGBD_PDL set in the
// environment, consecutive kernels are launched with programmatic stream
// serialization.  Every kernel starts with pdl_wait(), which then returns once
// the kernel it depends on has completed and its writes are visible; under an
// ordinary launch it returns at once.  Measured on the 1M-point frame it
// gained nothing (0.2635 vs 0.2632 ms), and letting the next kernel launch at
// the start of each kernel cost 12 us (waiting blocks held resources the
// multi-wave kernels needed), so ordinary launches are the default.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

bool pdl_enabled();  // true if the environment sets FGBD_PDL

// Launch `kernel` on `stream`: cooperative (all blocks resident, for the grid
// barriers) or with programmatic stream serialization.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                                 bool cooperative, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attrs[1];
  cfg.attrs = attrs;
  cfg.numAttrs = 0;
  if (cooperative) {
    attrs[0].id = cudaLaunchAttributeCooperative;
    attrs[0].val.cooperative = 1;
    cfg.numAttrs = 1;
  } else if (pdl_enabled()) {
    attrs[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attrs[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Run `set` (a kernel attribute change, which is idempotent) once per device:
// `done` holds one bit per device index.  Safe from several host threads; two
// threads may both run `set` the first time, which changes nothing.
template <typename F>
inline cudaError_t once_per_device(std::atomic<unsigned long long>& done, F&& set) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = set();
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// zero [p, p + words) on `stream` (a kernel, so it joins the programmatic chain)
cudaError_t launch_zero_words(uint32_t* p, size_t words, cudaStream_t stream);

}  // namespace fgbd
