// C ABI of the FGBD library (declared in include/fgbd.h).
//
// A context owns one device allocation sized for `capacity` points and
// carved into the buffers below.  Each ABI call validates its arguments on
// the host, enqueues kernels on the caller's stream and returns; device-side
// errors are latched in DevScalars::status and surfaced by the synchronising
// calls.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/fgbd.h"
#include "fgbd_internal.cuh"

using namespace fgbd;

struct fgbd_ctx {
  uint64_t uid = 0;  // unique over the process: a destroyed context's id never comes back
  int device = 0;
  int num_sms = 0;
  int filter_per_sm = 1;
  int64_t capacity = 0;
  fgbd_params params{};
  void* mem = nullptr;
  size_t mem_bytes = 0;
  DevScalars* sc = nullptr;
  SortBufs sb{};
  GraphBufs gb{};
  uint32_t* y8 = nullptr;
  float4* yf = nullptr;
  float* spread = nullptr;
  float4* x0 = nullptr;
  float4* x1 = nullptr;
  float4* xbest = nullptr;  // the global reading of the q search: the best iterate (else null)
  float4* w4 = nullptr;     // window 1: normalised Eq. 4 weights of the slots (FilterArgs::w4, w2)
  float2* w2 = nullptr;
  double* f64part = nullptr;
  int f64_blocks = 0;
  WideNe wne{};  // noise-estimate scratch of windows w > 1 (unused at window 1)
  int64_t* scan_tmp = nullptr;
  // state of the frame held in the context
  int n = 0;
  bool has_graph = false;
  bool has_noise = false;
  bool has_sel = false;
  const void* noise_rgb = nullptr;
  int noise_dtype = -1;
  std::string err;
  uint64_t graph_gen = 0;  // incremented by every graph build
  bool ever_selected = false;  // sc->q_sel holds a selected q (fgbd_run_reuse may use it)
  // differentiable filter: workspace (allocated by the first forward call that needs it) and the
  // state of the last forward call, which the backward call differentiates
  void* dmem = nullptr;
  size_t dmem_bytes = 0;
  DiffBufs db{};
  float4* d_ckpt = nullptr;   // x_0, x_c, x_2c, ... (c = checkpoint interval)
  float4* d_seg = nullptr;    // x_{t0+1} .. x_{t0+c-1} of one segment (backward)
  float4* d_pp[2] = {};       // ping-pong for steps and for the adjoint
  double* d_part = nullptr;   // per step and block: dL/dalpha, dL/dsigma terms
  int d_q = -1, d_c = 1, d_n = 0, d_grid = 0;
  float d_alpha = 0.5f;
  double d_sigma = 0.0;
  uint64_t d_gen = 0;
  bool d_valid = false;
  // filter steps stored by the noise-estimate launch (see filter_step.cuh)
  float4* spec_x = nullptr;   // [kSpecMax][cap]
  int32_t* spec_z = nullptr;  // [kSpecMax][cap]
  uint8_t* keep8 = nullptr;   // [cap]
  int spec_depth = 0;         // steps stored for noise_rgb on the current graph (0: none)
  // fgbd_run replays: CUDA graphs of whole runs, keyed by their arguments
  struct RunKey {
    const void* xyz;
    int64_t n;
    const void* rgb_in;
    int32_t in_dtype;
    void* rgb_out;
    int32_t out_dtype;
    bool operator==(const RunKey& o) const {
      return xyz == o.xyz && n == o.n && rgb_in == o.rgb_in && in_dtype == o.in_dtype && rgb_out == o.rgb_out &&
             out_dtype == o.out_dtype;
    }
  };
  struct RunGraph {
    RunKey key;
    cudaGraphExec_t exec;
    int64_t launches;
  };
  std::vector<RunGraph> run_graphs;  // most recent last
  std::vector<RunKey> run_seen;      // keys run once directly (the next call captures)
  // fgbd_run_batch replays (held by the batch's first context): per frame its
  // context and arguments, and the launches the capture counted for it
  struct BatchGraph {
    std::vector<fgbd_ctx*> ctxs;
    std::vector<uint64_t> uids;  // the contexts' ids: a graph of a destroyed context never matches
    std::vector<RunKey> keys;
    std::vector<int64_t> launches;
    BatchShape shape;            // the block shapes it was recorded with
    cudaGraphExec_t exec;
  };
  std::vector<BatchGraph> batch_graphs;  // most recent last
  std::vector<std::pair<std::vector<uint64_t>, std::vector<RunKey>>> batch_seen;
  cudaStream_t cap_stream = nullptr;
  bool graphs_on = true;
  // batched runs: this context's own stream and the events that order it
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr;    // recorded on the caller's stream (first context of a batch)
  cudaEvent_t ev_filter = nullptr;  // this frame's cooperative filter has finished
  cudaEvent_t ev_join = nullptr;    // all of this frame's work has finished
  // fgbd_run_host: two staging slots (coordinates, colours in, colours out) and
  // the copy streams and events that pipeline consecutive calls
  void* stage = nullptr;
  size_t stage_bytes = 0;
  int stage_next = 0;
  bool stage_used[2] = {false, false};
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t ev_in[2] = {}, ev_run[2] = {}, ev_out[2] = {};
  // instrumentation
  int64_t launches = 0;
  bool timing = false;
  cudaEvent_t ev[2 * FGBD_TIMING_CAP] = {};
  const char* ev_name[FGBD_TIMING_CAP] = {};
  int n_timed = 0;
};

// An exported graph: CSR in input order with the Eq. 4 weights (fgbd_graph_export).
struct fgbd_graph {
  int device = 0;
  int64_t n = 0;
  int64_t nnz = 0;
  double sigma_g = 0.0;
  void* mem = nullptr;
  int64_t* row_ptr = nullptr;
  int32_t* col = nullptr;
  float* w = nullptr;
};

namespace {

// NVTX range over one API call (header-only NVTX 3: no cost unless a profiler is attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
      changed = cudaSetDevice(dev) == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

fgbd_status cuda_fail(fgbd_ctx* ctx, cudaError_t e, const char* where) {
  if (ctx) {
    ctx->err = std::string(where) + ": " + cudaGetErrorString(e);
  }
  return FGBD_ECUDA;
}

#define FGBD_CUDA(ctx, expr)                                  \
  do {                                                        \
    const cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #expr);  \
  } while (0)

// Record one kernel launch: optional events around it, and the launch count.
struct LaunchScope {
  fgbd_ctx* ctx;
  cudaStream_t st;
  int slot = -1;
  LaunchScope(fgbd_ctx* c, const char* name, cudaStream_t s, int kernels = 1) : ctx(c), st(s) {
    ctx->launches += kernels;
    if (ctx->timing && ctx->n_timed < FGBD_TIMING_CAP) {
      slot = ctx->n_timed++;
      ctx->ev_name[slot] = name;
      cudaEventRecord(ctx->ev[2 * slot], st);
    }
  }
  ~LaunchScope() {
    if (slot >= 0) cudaEventRecord(ctx->ev[2 * slot + 1], st);
  }
};

#define FGBD_LAUNCH(ctx, name, st, expr)       \
  do {                                         \
    LaunchScope scope_(ctx, name, st);         \
    FGBD_CUDA(ctx, expr);                      \
  } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// distance between the C2 and C3 halves of ord23: a multiple of 64 points, so
// both halves start 256-byte aligned
int ord_stride(const fgbd_ctx* ctx) { return int(align_up(size_t(ctx->capacity), 64)); }

bool params_ok(const fgbd_params& p) {
  if (p.bits < 1 || p.bits > kMaxBits) return false;
  if (p.window < 1) return false;
  if (!(p.fslr_factor > 0.0) || p.fslr_factor > 1e30) return false;
  if (p.q_max < 0 || p.q_max > kQCap) return false;
  if (p.variant & ~(FGBD_VARIANT_NO_FSLR | FGBD_VARIANT_UNSORTED_PATCH | FGBD_VARIANT_SAME_LINE |
                    FGBD_VARIANT_SIGMA_NODE | FGBD_VARIANT_SIGMA_PAIR | FGBD_VARIANT_POOLED_PATCH |
                    FGBD_VARIANT_GLOBAL_Q))
    return false;
  if ((p.variant & FGBD_VARIANT_SIGMA_NODE) && (p.variant & FGBD_VARIANT_SIGMA_PAIR)) return false;
  if (p.flags & ~FGBD_FLAG_FUSED_SELECT) return false;
  for (int r : p.reserved)
    if (r != 0) return false;
  return true;
}

bool dtype_ok(int32_t d) { return d == FGBD_U8 || d == FGBD_F32; }

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

void zero_region(fgbd_ctx* ctx, size_t from, size_t to, cudaStream_t st, cudaError_t* e) {
  if (*e != cudaSuccess) return;
  if (to > from) ctx->launches += 1;  // one k_zero_words launch
  *e = launch_zero_words(reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(ctx->sc) + from), (to - from) / 4, st);
}

fgbd_status take_device_status(fgbd_ctx* ctx, cudaStream_t st) {
  uint32_t status = 0;
  FGBD_CUDA(ctx, cudaStreamSynchronize(st));
  FGBD_CUDA(ctx, cudaMemcpy(&status, &ctx->sc->status, sizeof(status), cudaMemcpyDeviceToHost));
  if (status) {
    const uint32_t zero = 0;
    FGBD_CUDA(ctx, cudaMemcpy(&ctx->sc->status, &zero, sizeof(zero), cudaMemcpyHostToDevice));
    if (status & kFlagTimeout) return FGBD_ETIMEOUT;
    if (status & kFlagRange) return FGBD_ERANGE;
  }
  return FGBD_OK;
}

FilterArgs filter_args(fgbd_ctx* ctx, int mode, int q_fixed, const double* sigma_src, void* out,
                       int out_dtype, int dtype) {
  FilterArgs a{};
  a.n = ctx->n;
  a.bits = ctx->params.bits;
  a.dtype = dtype;
  a.mode = mode;
  a.q_fixed = q_fixed;
  a.q_max = ctx->params.q_max;
  a.fslr_factor = ctx->params.fslr_factor;
  a.all_points = (ctx->params.variant & FGBD_VARIANT_NO_FSLR) != 0;
  a.sigma_src = sigma_src ? sigma_src : &ctx->sc->sigma_est;
  a.y8 = ctx->y8;
  a.yf = ctx->yf;
  a.spread = ctx->spread;
  a.pk = ctx->gb.pk;
  a.c4 = ctx->gb.c4;
  a.rank1 = ctx->gb.rank1;
  a.xbuf0 = ctx->x0;
  a.xbuf1 = ctx->x1;
  a.out = out;
  a.out_dtype = out_dtype;
  a.sc = ctx->sc;
  a.spec_depth = 0;
  a.spec_x = ctx->spec_x;
  a.spec_z = ctx->spec_z;
  a.cap = int(align_up(size_t(ctx->capacity), 64));  // row stride of spec_x / spec_z
  a.keep8 = ctx->keep8;
  a.cx = ctx->gb.cx;
  a.nx = ctx->gb.nx;
  a.cx_stride = ctx->gb.cx_stride;
  a.node_sig = (ctx->params.variant & FGBD_VARIANT_SIGMA_PAIR) ? ctx->gb.node_sig : nullptr;
  a.q_global = (ctx->params.variant & FGBD_VARIANT_GLOBAL_Q) ? 1 : 0;
  a.xbest = ctx->xbest;
  a.w4 = ctx->w4;
  a.w2 = ctx->w2;
  return a;
}

int filter_grid_for(const fgbd_ctx* ctx, int n) {
  const int need = std::max(1, (n + kFilterThreads - 1) / kFilterThreads);
  return std::max(1, std::min(need, ctx->filter_per_sm * ctx->num_sms));
}

// Carve the differentiable-filter workspace for n points, q steps, checkpoint
// interval c; grow the allocation if needed (this synchronises the device).
fgbd_status diff_workspace(fgbd_ctx* ctx, int n, int q, int c, int grid) {
  const size_t N = size_t(std::max(n, 1));
  const size_t nck = size_t(q / c + 1);
  const size_t sizes[] = {N * kK * 4, N * kK * 4, N * kK * 4, N * kK * 4, N * 4,  // nb, R, RT, d2, e
                          nck * N * 16, size_t(c > 1 ? c - 1 : 1) * N * 16,     // checkpoints, segment
                          N * 16, N * 16,                                       // ping-pong
                          size_t(std::max(q, 1)) * size_t(grid) * 2 * 8};       // partials
  size_t total = 0;
  for (size_t b : sizes) total = align_up(total, 256) + b;
  total = align_up(total, 256);
  if (total > ctx->dmem_bytes) {
    if (ctx->dmem) {
      cudaDeviceSynchronize();
      cudaFree(ctx->dmem);
      ctx->dmem = nullptr;
      ctx->dmem_bytes = 0;
    }
    if (cudaMalloc(&ctx->dmem, total) != cudaSuccess) {
      cudaGetLastError();
      ctx->dmem = nullptr;
      return FGBD_ENOMEM;
    }
    ctx->dmem_bytes = total;
  }
  char* base = static_cast<char*>(ctx->dmem);
  size_t off = 0;
  void* ptrs[10];
  for (int k = 0; k < 10; ++k) {
    off = align_up(off, 256);
    ptrs[k] = base + off;
    off += sizes[k];
  }
  ctx->db.nb = static_cast<int32_t*>(ptrs[0]);
  ctx->db.R = static_cast<float*>(ptrs[1]);
  ctx->db.RT = static_cast<float*>(ptrs[2]);
  ctx->db.d2 = static_cast<float*>(ptrs[3]);
  ctx->db.e = static_cast<float*>(ptrs[4]);
  ctx->d_ckpt = static_cast<float4*>(ptrs[5]);
  ctx->d_seg = static_cast<float4*>(ptrs[6]);
  ctx->d_pp[0] = static_cast<float4*>(ptrs[7]);
  ctx->d_pp[1] = static_cast<float4*>(ptrs[8]);
  ctx->d_part = static_cast<double*>(ptrs[9]);
  return FGBD_OK;
}

void release_batch_objects(fgbd_ctx* ctx) {
  for (cudaEvent_t* e : {&ctx->ev_fork, &ctx->ev_filter, &ctx->ev_join})
    if (*e) {
      cudaEventDestroy(*e);
      *e = nullptr;
    }
  for (auto& g : ctx->run_graphs) cudaGraphExecDestroy(g.exec);
  ctx->run_graphs.clear();
  for (auto& g : ctx->batch_graphs) cudaGraphExecDestroy(g.exec);
  ctx->batch_graphs.clear();
  for (cudaStream_t* st : {&ctx->side, &ctx->cap_stream})
    if (*st) {
      cudaStreamDestroy(*st);
      *st = nullptr;
    }
}

// `zeroed`: the caller has already zeroed the scalar regions this call fills.
// `rgb_gather` (fgbd_run): the colours of the frame, gathered into sorted order
// on the context's side stream as soon as the C1 order exists, beside the C2
// pass and the link step, which do not touch them (do_estimate then joins it).
fgbd_status do_build(fgbd_ctx* ctx, const int32_t* xyz, int64_t n64, cudaStream_t st, bool zeroed = false,
                     const void* rgb_gather = nullptr, int32_t gather_dtype = FGBD_U8) {
  if (n64 < 0 || n64 > ctx->capacity) return FGBD_EINVAL;
  if (n64 > 0 && !xyz) return FGBD_EINVAL;
  const int n = int(n64);
  const int bits = ctx->params.bits;
  ctx->has_graph = ctx->has_noise = ctx->has_sel = false;
  ctx->spec_depth = 0;
  ctx->noise_rgb = nullptr;
  ctx->n = n;
  ctx->graph_gen += 1;
  cudaError_t e = cudaSuccess;
  if (!zeroed) zero_region(ctx, offsetof(DevScalars, n_edges), offsetof(DevScalars, build_end_), st, &e);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "memset");
  if (n > 0) {
    // kernel names carry the pass: 0 = y-slabs, 1 = C1 (on z, over C3), 2 = C2 (on x, over C1)
    static const char* const kCounts[kSlgPasses] = {"slg_counts0", "slg_counts1", "slg_counts2"};
    static const char* const kScan[kSlgPasses] = {"slg_scan0", "slg_scan1", "slg_scan2"};
    static const char* const kScatter[kSlgPasses] = {"slg_scatter0", "slg_scatter1", "slg_scatter2"};
    FGBD_LAUNCH(ctx, "slg_hist", st, launch_coord_hist(xyz, n, bits, ctx->sc, &ctx->sb, ctx->num_sms, st));
    for (int p = 0; p < kSlgPasses; ++p) {
      const SortPassArgs a = slg_pass_args(p, xyz, n, bits, ord_stride(ctx), ctx->sb, ctx->gb, ctx->sc);
      if (!pass_counted_before(p)) FGBD_LAUNCH(ctx, kCounts[p], st, launch_tile_counts(a, st));
      FGBD_LAUNCH(ctx, kScan[p], st, launch_tile_scan(a, st));
      FGBD_LAUNCH(ctx, kScatter[p], st, launch_sort_scatter(a, st));
      if (p == 0)
        FGBD_LAUNCH(ctx, "slg_slab", st,
                    launch_slab_sort(n, bits, ord_stride(ctx), ctx->sb, ctx->gb, ctx->sc, st));
      if (p == 1 && rgb_gather) {
        FGBD_CUDA(ctx, cudaEventRecord(ctx->ev_fork, st));
        FGBD_CUDA(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0));
        FGBD_LAUNCH(ctx, "gather_colors", ctx->side,
                    launch_gather_colors(rgb_gather, gather_dtype, n, ctx->gb.perm1, ctx->y8, ctx->yf, ctx->side));
        FGBD_CUDA(ctx, cudaEventRecord(ctx->ev_join, ctx->side));
      }
    }
    const bool same_line = (ctx->params.variant & FGBD_VARIANT_SAME_LINE) != 0;
    if (ctx->params.window == 1)
      FGBD_LAUNCH(ctx, "slg_link", st,
                  launch_link(n, bits, ord_stride(ctx), same_line, ctx->gb, ctx->sb, ctx->sc, ctx->num_sms, st));
    else
      FGBD_LAUNCH(ctx, "slg_link", st,
                  launch_link_wide(n, bits, ord_stride(ctx), ctx->params.window, same_line, ctx->gb, ctx->sb,
                                   ctx->sc, ctx->num_sms, st));
    if (same_line) ctx->launches += 1;  // and k_c1_line_flags
    if (ctx->params.variant & (FGBD_VARIANT_SIGMA_NODE | FGBD_VARIANT_SIGMA_PAIR))
      FGBD_LAUNCH(ctx, "slg_node_sigma", st,
                  launch_node_sigma(n, bits, ctx->gb, ctx->sc, ctx->num_sms, st));
  }
  ctx->has_graph = true;
  return FGBD_OK;
}

// With `fuse`, the estimate launch also selects q and writes the filtered
// colours to fuse_out (what do_select with the estimated sigma would do).
fgbd_status do_estimate(fgbd_ctx* ctx, const void* rgb, int32_t dtype, double* sigma_out, cudaStream_t st,
                        bool speculate = true, bool fuse = false, void* fuse_out = nullptr,
                        int32_t fuse_out_dtype = FGBD_U8, bool zeroed = false, bool pregathered = false) {
  if (!ctx->has_graph) return FGBD_ESTATE;
  if (!dtype_ok(dtype)) return FGBD_EINVAL;
  if (ctx->n > 0 && !rgb) return FGBD_EINVAL;
  const int n = ctx->n;
  ctx->has_noise = ctx->has_sel = false;
  cudaError_t e = cudaSuccess;
  if (!zeroed) zero_region(ctx, offsetof(DevScalars, n_patches), offsetof(DevScalars, ne_end_), st, &e);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "memset");
  if (ctx->params.window > 1) {
    // wider windows: moments, their reduction, the eigenvector block, the Rayleigh
    // quotients with the tail rule; no filter steps are taken beside them
    if (n > 0) {
      if (pregathered)
        FGBD_CUDA(ctx, cudaStreamWaitEvent(st, ctx->ev_join, 0));
      else
        FGBD_LAUNCH(ctx, "gather_colors", st,
                    launch_gather_colors(rgb, dtype, n, ctx->gb.perm1, ctx->y8, ctx->yf, st));
    }
    static const char* const kStage[4] = {"ne_wide_moments", "ne_wide_reduce", "ne_wide_eigvec", "ne_wide_tail"};
    for (int stage = n > 0 ? 0 : 1; stage < 4; ++stage)
      FGBD_LAUNCH(ctx, kStage[stage], st,
                  launch_ne_wide(stage, n, ctx->params.bits, ctx->params.window, dtype, ctx->gb, ctx->y8, ctx->yf,
                                 ctx->spread, ctx->wne, ctx->sc, sigma_out, ctx->num_sms, st));
    ctx->spec_depth = 0;
    ctx->has_noise = true;
    ctx->noise_rgb = rgb;
    ctx->noise_dtype = dtype;
    return FGBD_OK;
  }
  int nblocks = 0;
  if (n > 0) {
    if (pregathered)
      FGBD_CUDA(ctx, cudaStreamWaitEvent(st, ctx->ev_join, 0));  // the gather do_build started
    else
      FGBD_LAUNCH(ctx, "gather_colors", st,
                  launch_gather_colors(rgb, dtype, n, ctx->gb.perm1, ctx->y8, ctx->yf, st));
    nblocks = ne_moment_blocks(n, ctx->num_sms);
    // (with x_0 of the filter steps into ctx->x0, which step 1 then reads as one 16-byte load a point)
    FGBD_LAUNCH(ctx, "ne_moments", st,
                launch_ne_moments(n, ctx->params.bits, dtype, ctx->gb, ctx->y8, ctx->yf, ctx->spread, ctx->f64part,
                                  ctx->sc, ctx->num_sms, true,
                                  (ctx->params.variant & FGBD_VARIANT_UNSORTED_PATCH) == 0, st,
                                  speculate ? ctx->x0 : nullptr));
  }
  // the same launch stores the first filter steps of these colours on the other SMs
  FilterArgs spec = filter_args(ctx, 0, 0, nullptr, fuse ? fuse_out : nullptr, fuse ? fuse_out_dtype : 0, dtype);
  spec.spec_depth = speculate ? std::min(kSpecMax, int(ctx->params.q_max)) : 0;
  spec.x0 = speculate && n > 0 ? ctx->x0 : nullptr;
  ctx->spec_depth = n > 0 && ctx->num_sms >= 2 ? spec.spec_depth : 0;
  const bool fused = fuse && ctx->spec_depth > 0;
  spec.fuse = fused ? 1 : 0;
  if (fused && !zeroed) {
    zero_region(ctx, offsetof(DevScalars, ysq_keep), offsetof(DevScalars, sel_end_), st, &e);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "memset");
  }
  FGBD_LAUNCH(ctx, "ne_finalize", st,
              launch_ne_finalize(dtype, ctx->f64part, nblocks, ctx->sc, sigma_out, &spec, ctx->num_sms, st));
  ctx->has_noise = true;
  ctx->noise_rgb = rgb;
  ctx->noise_dtype = dtype;
  if (fused) {
    ctx->has_sel = true;
    ctx->ever_selected = true;
  }
  return FGBD_OK;
}

fgbd_status do_select(fgbd_ctx* ctx, const void* rgb, int32_t dtype, const double* sigma_est, int32_t* q_out,
                      void* out, int32_t out_dtype, cudaStream_t st, bool zeroed = false) {
  if (!ctx->has_noise) return FGBD_ESTATE;
  if (!dtype_ok(dtype)) return FGBD_EINVAL;
  if (rgb != ctx->noise_rgb || dtype != ctx->noise_dtype) return FGBD_ESTATE;
  ctx->has_sel = false;
  cudaError_t e = cudaSuccess;
  if (!zeroed) zero_region(ctx, offsetof(DevScalars, ysq_keep), offsetof(DevScalars, sel_end_), st, &e);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "memset");
  FilterArgs a = filter_args(ctx, 0, 0, sigma_est, out, out_dtype, dtype);
  a.spec_depth = ctx->spec_depth;  // the kernel checks that they were all stored
  FGBD_LAUNCH(ctx, "filter_select", st, launch_filter(a, filter_grid_for(ctx, ctx->n), st));
  if (q_out) FGBD_CUDA(ctx, cudaMemcpyAsync(q_out, &ctx->sc->q_sel, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  ctx->has_sel = true;
  ctx->ever_selected = true;
  return FGBD_OK;
}

fgbd_status direct_run(fgbd_ctx* ctx, const fgbd_ctx::RunKey& k, cudaStream_t st) {
  if (k.n < 0 || k.n > ctx->capacity) return FGBD_EINVAL;
  // the build, noise and selection regions of the scalars are adjacent: one launch zeroes them
  cudaError_t e = cudaSuccess;
  zero_region(ctx, offsetof(DevScalars, n_edges), offsetof(DevScalars, sel_end_), st, &e);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "memset");
  fgbd_status s = do_build(ctx, static_cast<const int32_t*>(k.xyz), k.n, st, true, k.rgb_in, k.in_dtype);
  if (s != FGBD_OK) return s;
  // with FGBD_FLAG_FUSED_SELECT the estimate launch selects and filters too
  const bool fuse = (ctx->params.flags & FGBD_FLAG_FUSED_SELECT) != 0 && ctx->params.window == 1;
  s = do_estimate(ctx, k.rgb_in, k.in_dtype, nullptr, st, true, fuse, k.rgb_out, k.out_dtype, true, k.n > 0);
  if (s != FGBD_OK) return s;
  if (ctx->has_sel) return FGBD_OK;
  return do_select(ctx, k.rgb_in, k.in_dtype, nullptr, nullptr, k.rgb_out, k.out_dtype, st, true);
}

// host state after a replayed run: what a direct run of the same arguments leaves
void mark_run_done(fgbd_ctx* ctx, const fgbd_ctx::RunKey& k, int64_t launches) {
  ctx->n = int(k.n);
  ctx->graph_gen += 1;
  ctx->has_graph = ctx->has_noise = ctx->has_sel = true;
  ctx->ever_selected = true;
  ctx->noise_rgb = k.rgb_in;
  ctx->noise_dtype = k.in_dtype;
  ctx->launches += launches;
}

// Record a run of these arguments into a CUDA graph (on the context's own
// stream, so the caller's stream is never in capture mode), then launch it on
// the caller's stream.  If the capture fails for any reason the run is made
// directly and the context stops capturing.
fgbd_status capture_run(fgbd_ctx* ctx, const fgbd_ctx::RunKey& k, cudaStream_t st) {
  const cudaStream_t cs = ctx->cap_stream;
  const int64_t launches0 = ctx->launches;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // the captured work must follow everything already on the caller's stream
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    ctx->graphs_on = false;
    return direct_run(ctx, k, st);
  }
  const fgbd_status s = direct_run(ctx, k, cs);
  const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
  bool ok = s == FGBD_OK && ce == cudaSuccess && graph;
  ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    cudaGetLastError();
    if (exec) cudaGraphExecDestroy(exec);
    ctx->launches = launches0;
    ctx->graphs_on = false;
    if (s != FGBD_OK && s != FGBD_ECUDA) return s;
    return direct_run(ctx, k, st);
  }
  FGBD_CUDA(ctx, cudaGraphLaunch(exec, st));
  if (ctx->run_graphs.size() >= 8) {
    cudaGraphExecDestroy(ctx->run_graphs.front().exec);
    ctx->run_graphs.erase(ctx->run_graphs.begin());
  }
  ctx->run_graphs.push_back({k, exec, ctx->launches - launches0});
  return FGBD_OK;
}

// ---------------------------------------------------------------- segmented batches
// A batch whose frames share the window (1), the ablation switches and the
// colour type runs each stage as one launch over up to kSegMax frames
// (segmented launches, fgbd_internal.cuh): 15 launches for the whole chunk
// instead of 15 per frame, every frame's short latency-bound kernels
// side by side in one grid, the estimate launch with one eigen block per
// frame, and one cooperative selection/filter for all frames (each frame's
// blocks synchronise among themselves).  Each frame's blocks run the same
// code with the same block counts as its one-frame kernels (or, for the
// block shapes the tuner may change, code whose results do not depend on the
// shape), so the outputs equal fgbd_run's bit for bit.

bool seg_eligible(const std::vector<fgbd_ctx*>& ctxs, const std::vector<fgbd_ctx::RunKey>& keys) {
  const fgbd_ctx* c0 = ctxs[0];
  if (c0->num_sms < 2 * kSegMax) return false;
  for (size_t f = 0; f < ctxs.size(); ++f) {
    const fgbd_ctx* c = ctxs[f];
    if (c->params.window != 1 || c->params.variant != c0->params.variant || c->num_sms != c0->num_sms) return false;
    // the readings that add a kernel or a buffer run on streams
    if (c->params.variant & (FGBD_VARIANT_SIGMA_NODE | FGBD_VARIANT_SIGMA_PAIR | FGBD_VARIANT_POOLED_PATCH |
                             FGBD_VARIANT_GLOBAL_Q))
      return false;
    if (keys[f].in_dtype != keys[0].in_dtype || keys[f].n < 1) return false;
  }
  return true;
}

// Frames [i0, i1) of the batch (i1 - i0 <= kSegMax), enqueued on `st`.
fgbd_status seg_chunk(const std::vector<fgbd_ctx*>& ctxs, const std::vector<fgbd_ctx::RunKey>& keys, int i0,
                      int i1, const BatchShape& shape, cudaStream_t st) {
  const int F = i1 - i0;
  fgbd_ctx* lead = ctxs[i0];
  const int num_sms = lead->num_sms;
  const int dtype = keys[i0].in_dtype;
  const bool same_line = (lead->params.variant & FGBD_VARIANT_SAME_LINE) != 0;
  const bool sorted = (lead->params.variant & FGBD_VARIANT_UNSORTED_PATCH) == 0;
  ZeroArgs z[kSegMax];
  HistArgs h[kSegMax];
  LinkArgs l[kSegMax];
  GatherArgs g[kSegMax];
  MomentArgs m[kSegMax];
  FilterArgs spec[kSegMax], sel[kSegMax];
  const double* f64[kSegMax];
  int nblk[kSegMax], ns[kSegMax], bits[kSegMax], caps[kSegMax];
  SortBufs sbs[kSegMax];
  GraphBufs gbs[kSegMax];
  DevScalars* scs[kSegMax];
  for (int f = 0; f < F; ++f) {
    fgbd_ctx* c = ctxs[i0 + f];
    const fgbd_ctx::RunKey& k = keys[i0 + f];
    const int n = int(k.n);
    const int32_t* xyz = static_cast<const int32_t*>(k.xyz);
    ns[f] = n;
    bits[f] = c->params.bits;
    caps[f] = ord_stride(c);
    sbs[f] = c->sb;
    gbs[f] = c->gb;
    scs[f] = c->sc;
    z[f] = ZeroArgs{reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(c->sc) + offsetof(DevScalars, n_edges)),
                    (offsetof(DevScalars, sel_end_) - offsetof(DevScalars, n_edges)) / 4};
    h[f] = hist_args(xyz, n, bits[f], c->sc, c->sb);
    l[f] = link_args(n, bits[f], caps[f], c->gb, c->sb, c->sc);
    g[f] = GatherArgs{k.rgb_in, dtype, n, c->gb.perm1, c->y8, c->yf};
    m[f] = moment_args(n, bits[f], c->gb, c->y8, c->yf, c->spread, c->f64part, true, sorted, c->sc);
    // the state fgbd_run's calls leave (n is set first: filter_args reads it)
    c->n = n;
    spec[f] = filter_args(c, 0, 0, nullptr, nullptr, 0, dtype);
    spec[f].spec_depth = std::min(kSpecMax, int(c->params.q_max));
    sel[f] = filter_args(c, 0, 0, nullptr, k.rgb_out, k.out_dtype, dtype);
    sel[f].spec_depth = spec[f].spec_depth;
    f64[f] = c->f64part;
    nblk[f] = ne_moment_blocks(n, num_sms);
  }
  FGBD_LAUNCH(lead, "seg_zero", st, launch_zero_words_seg(z, F, st));
  FGBD_LAUNCH(lead, "seg_hist", st, launch_coord_hist_seg(h, F, num_sms, st));
  static const char* const kPass[kSlgPasses][3] = {{"seg_counts0", "seg_scan0", "seg_scatter0"},
                                                   {"seg_counts1", "seg_scan1", "seg_scatter1"},
                                                   {"seg_counts2", "seg_scan2", "seg_scatter2"}};
  for (int p = 0; p < kSlgPasses; ++p) {
    SortPassArgs a[kSegMax];
    for (int f = 0; f < F; ++f) {
      fgbd_ctx* c = ctxs[i0 + f];
      a[f] = slg_pass_args(p, static_cast<const int32_t*>(keys[i0 + f].xyz), ns[f], bits[f], caps[f], c->sb, c->gb,
                           c->sc);
    }
    {
      // (counts,) scan and scatter: two or three launches under one timing scope
      LaunchScope scope_(lead, kPass[p][2], st, pass_counted_before(p) ? 2 : 3);
      FGBD_CUDA(lead, launch_sort_pass_seg(a, F, shape.scatter_threads, st));
    }
    if (p == 0) FGBD_LAUNCH(lead, "seg_slab", st, launch_slab_sort_seg(ns, bits, caps, sbs, gbs, scs, F, st));
  }
  FGBD_LAUNCH(lead, "seg_link", st, launch_link_seg(l, F, same_line, num_sms, st));
  if (same_line) lead->launches += 1;  // and the line flags
  FGBD_LAUNCH(lead, "seg_gather", st, launch_gather_colors_seg(g, F, st));
  FGBD_LAUNCH(lead, "seg_moments", st, launch_ne_moments_seg(m, F, dtype, num_sms, st));
  FGBD_LAUNCH(lead, "seg_estimate", st, launch_ne_finalize_seg(spec, f64, nblk, F, num_sms, st));
  FGBD_LAUNCH(lead, "seg_select", st,
              launch_filter_seg(sel, F, shape.filter_threads, shape.filter_per_sm, num_sms, st));
  for (int f = 0; f < F; ++f) {
    fgbd_ctx* c = ctxs[i0 + f];
    mark_run_done(c, keys[i0 + f], 0);
    c->spec_depth = spec[f].spec_depth;
  }
  return FGBD_OK;
}

fgbd_status segmented_batch(const std::vector<fgbd_ctx*>& ctxs, const std::vector<fgbd_ctx::RunKey>& keys,
                            const BatchShape& shape, cudaStream_t st) {
  const int count = int(ctxs.size());
  const int chunk = std::max(1, std::min(shape.seg_frames, kSegMax));
  for (int i0 = 0; i0 < count; i0 += chunk) {
    const fgbd_status s = seg_chunk(ctxs, keys, i0, std::min(count, i0 + chunk), shape, st);
    if (s != FGBD_OK) return s;
  }
  return FGBD_OK;
}

// Block shapes of segmented batches, per device and frame-size class
// (floor(log2(mean points per frame))): set by fgbd_tune_batch or
// fgbd_set_batch_shape, the defaults otherwise.
struct TunedShape {
  int device;
  int size_class;
  BatchShape shape;
};
std::mutex g_shape_mutex;
std::vector<TunedShape> g_shapes;

int size_class(const std::vector<fgbd_ctx::RunKey>& keys) {
  double total = 0.0;
  for (const auto& k : keys) total += double(std::max<int64_t>(k.n, 1));
  const double mean = total / double(std::max<size_t>(keys.size(), 1));
  return int(std::floor(std::log2(std::max(mean, 1.0))));
}

// Untuned: segmented launches of up to kSegMax frames for frames below 2^18
// points, whose stages are short and whose working sets (about 180 bytes a
// point) fit the L2 together; per-frame streams above, where a frame's own
// working set fills the L2 and running the frames stage by stage would evict
// each frame's data between its stages (measured on 16 frames of 200k-1.2M
// points: 4.41 ms segmented against 3.45 ms on streams).
BatchShape default_shape(int cls) {
  BatchShape b;
  b.seg_frames = cls < 18 ? kSegMax : 0;
  return b;
}

BatchShape shape_for(int device, int cls) {
  std::lock_guard<std::mutex> lock(g_shape_mutex);
  for (const TunedShape& t : g_shapes)
    if (t.device == device && t.size_class == cls) return t.shape;
  return default_shape(cls);
}

void store_shape(int device, int cls, const BatchShape* shape) {
  std::lock_guard<std::mutex> lock(g_shape_mutex);
  for (size_t i = 0; i < g_shapes.size(); ++i) {
    if (g_shapes[i].device == device && g_shapes[i].size_class == cls) {
      if (shape) g_shapes[i].shape = *shape;
      else g_shapes.erase(g_shapes.begin() + long(i));
      return;
    }
  }
  if (shape) g_shapes.push_back({device, cls, *shape});
}

bool shape_ok(const BatchShape& b) {
  return b.seg_frames >= 0 && b.seg_frames <= kSegMax &&
         (b.scatter_threads == 256 || b.scatter_threads == 512 || b.scatter_threads == 1024) &&
         (b.filter_threads == 256 || b.filter_threads == 512) && b.filter_per_sm >= 1 && b.filter_per_sm <= 8;
}

// The batch of fgbd_run_batch, enqueued directly: segmented when the frames
// allow it, else every frame on its context's own stream, forked from `st`
// and joined back into it, the selection/filter launches (cooperative, each
// using the whole GPU) one frame after another.
fgbd_status stream_batch(const std::vector<fgbd_ctx*>& ctxs, const std::vector<fgbd_ctx::RunKey>& keys,
                         cudaStream_t st);

fgbd_status direct_batch(const std::vector<fgbd_ctx*>& ctxs, const std::vector<fgbd_ctx::RunKey>& keys,
                         const BatchShape& shape, cudaStream_t st) {
  if (shape.seg_frames > 0 && seg_eligible(ctxs, keys)) return segmented_batch(ctxs, keys, shape, st);
  return stream_batch(ctxs, keys, st);
}

fgbd_status stream_batch(const std::vector<fgbd_ctx*>& ctxs, const std::vector<fgbd_ctx::RunKey>& keys,
                         cudaStream_t st) {
  const int count = int(ctxs.size());
  fgbd_ctx* lead = ctxs[0];
  // fork: every frame's stream starts after the caller's earlier work
  FGBD_CUDA(lead, cudaEventRecord(lead->ev_fork, st));
  for (int f = 0; f < count; ++f) FGBD_CUDA(ctxs[f], cudaStreamWaitEvent(ctxs[f]->side, lead->ev_fork, 0));
  // graph and noise estimate of every frame, concurrently
  for (int f = 0; f < count; ++f) {
    fgbd_ctx* c = ctxs[f];
    const fgbd_ctx::RunKey& k = keys[f];
    fgbd_status s = do_build(c, static_cast<const int32_t*>(k.xyz), k.n, c->side);
    if (s == FGBD_OK) s = do_estimate(c, k.rgb_in, k.in_dtype, nullptr, c->side, false);
    if (s != FGBD_OK) return s;
  }
  // selection + filter: cooperative launches, one at a time (frame f waits for
  // frame f - 1's) so that two of them never compete for residency
  for (int f = 0; f < count; ++f) {
    fgbd_ctx* c = ctxs[f];
    const fgbd_ctx::RunKey& k = keys[f];
    if (f > 0) FGBD_CUDA(c, cudaStreamWaitEvent(c->side, ctxs[f - 1]->ev_filter, 0));
    const fgbd_status s = do_select(c, k.rgb_in, k.in_dtype, nullptr, nullptr, k.rgb_out, k.out_dtype, c->side);
    if (s != FGBD_OK) return s;
    FGBD_CUDA(c, cudaEventRecord(c->ev_filter, c->side));
  }
  // join: the caller's stream continues after every frame
  for (int f = 0; f < count; ++f) {
    FGBD_CUDA(ctxs[f], cudaEventRecord(ctxs[f]->ev_join, ctxs[f]->side));
    FGBD_CUDA(ctxs[f], cudaStreamWaitEvent(st, ctxs[f]->ev_join, 0));
  }
  return FGBD_OK;
}

// Record the batch into a CUDA graph on the first context's capture stream (the
// frames' own streams join the capture through the fork event), then launch it.
// If the capture fails the batch runs directly and the first context stops capturing.
fgbd_status capture_batch(fgbd_ctx* lead, const std::vector<fgbd_ctx*>& ctxs,
                          const std::vector<fgbd_ctx::RunKey>& keys, const BatchShape& shape, cudaStream_t st) {
  const cudaStream_t cs = lead->cap_stream;
  std::vector<int64_t> launches0;
  for (fgbd_ctx* c : ctxs) launches0.push_back(c->launches);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    lead->graphs_on = false;
    return direct_batch(ctxs, keys, shape, st);
  }
  const fgbd_status s = direct_batch(ctxs, keys, shape, cs);
  const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
  bool ok = s == FGBD_OK && ce == cudaSuccess && graph;
  ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    cudaGetLastError();
    if (exec) cudaGraphExecDestroy(exec);
    for (size_t f = 0; f < ctxs.size(); ++f) ctxs[f]->launches = launches0[f];
    lead->graphs_on = false;
    if (s != FGBD_OK && s != FGBD_ECUDA) return s;
    return direct_batch(ctxs, keys, shape, st);
  }
  FGBD_CUDA(lead, cudaGraphLaunch(exec, st));
  if (lead->batch_graphs.size() >= 4) {
    cudaGraphExecDestroy(lead->batch_graphs.front().exec);
    lead->batch_graphs.erase(lead->batch_graphs.begin());
  }
  fgbd_ctx::BatchGraph bg{ctxs, {}, keys, {}, shape, exec};
  for (fgbd_ctx* c : ctxs) bg.uids.push_back(c->uid);
  for (size_t f = 0; f < ctxs.size(); ++f) bg.launches.push_back(ctxs[f]->launches - launches0[f]);
  lead->batch_graphs.push_back(bg);
  return FGBD_OK;
}

}  // namespace

extern "C" {

int32_t fgbd_abi_version(void) { return FGBD_ABI_VERSION; }

const char* fgbd_status_str(fgbd_status s) {
  switch (s) {
    case FGBD_OK: return "FGBD_OK";
    case FGBD_EINVAL: return "FGBD_EINVAL: invalid argument";
    case FGBD_ERANGE: return "FGBD_ERANGE: coordinate outside [0, 2^bits)";
    case FGBD_ENOMEM: return "FGBD_ENOMEM: device allocation failed";
    case FGBD_ECUDA: return "FGBD_ECUDA: CUDA runtime error";
    case FGBD_ETIMEOUT: return "FGBD_ETIMEOUT: a bounded device wait gave up";
    case FGBD_ESTATE: return "FGBD_ESTATE: calls out of order";
    case FGBD_ENOTIMPL: return "FGBD_ENOTIMPL: not implemented";
  }
  return "unknown fgbd_status";
}

fgbd_status fgbd_params_default(fgbd_params* p) {
  if (!p) return FGBD_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->bits = 10;
  p->window = 1;
  p->fslr_factor = 2.0;
  p->q_max = 64;
  return FGBD_OK;
}

fgbd_status fgbd_ctx_create(int64_t capacity, const fgbd_params* params, fgbd_ctx** out) {
  if (!out) return FGBD_EINVAL;
  *out = nullptr;
  if (capacity < 1 || capacity >= (int64_t(1) << 30)) return FGBD_EINVAL;
  fgbd_params p;
  if (params) p = *params;
  else fgbd_params_default(&p);
  if (!params_ok(p)) return FGBD_EINVAL;
  // windows 2..3 are built; the unsorted-patch ablation is defined for window 1 only,
  // and the pair bandwidths and pooled patches are built for window 1 only
  if (p.window > kMaxWindow) return FGBD_ENOTIMPL;
  if (p.window > 1 && (p.variant & (FGBD_VARIANT_UNSORTED_PATCH | FGBD_VARIANT_SIGMA_PAIR | FGBD_VARIANT_POOLED_PATCH)))
    return FGBD_ENOTIMPL;
  fgbd_ctx* ctx = new (std::nothrow) fgbd_ctx();
  if (!ctx) return FGBD_ENOMEM;
  static std::atomic<uint64_t> next_uid{1};
  ctx->uid = next_uid.fetch_add(1);
  ctx->capacity = capacity;
  ctx->params = p;
  if (cudaGetDevice(&ctx->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
    delete ctx;
    return FGBD_ECUDA;
  }
  const int nx = extra_slots(p.window);
  ctx->filter_per_sm = std::max(1, filter_grid(1 << 30, ctx->num_sms, nx) / ctx->num_sms);

  const size_t C = size_t(capacity);
  const int tiles = int((C + kSortTile - 1) / kSortTile);
  ctx->f64_blocks = ne_moment_blocks(int(C), ctx->num_sms);
  const size_t kP = size_t(kD) * kD + kD + 1;
  // wider windows: the further neighbour slots and the noise-estimate scratch
  const bool wide = p.window > 1;
  const size_t wD = size_t(3 * (6 * p.window + 1));
  const int w_blocks = ne_wide_blocks(int(C), ctx->num_sms);
  const size_t wP = ne_wide_part_entries(p.window);
  struct Item {
    void** ptr;
    size_t bytes;
  };
  void* keys0 = nullptr;
  void* keys1 = nullptr;
  void* vals0 = nullptr;
  void* vals1 = nullptr;
  const Item items[] = {
      {reinterpret_cast<void**>(&ctx->sc), sizeof(DevScalars)},
      {&keys0, C * 4},
      {&keys1, C * 4},
      {&vals0, C * 4},
      {&vals1, C * 4},
      {reinterpret_cast<void**>(&ctx->sb.tile_counts), size_t(kSlgPasses) * kMaxRadix * tiles * 4},
      {reinterpret_cast<void**>(&ctx->gb.perm1), C * 4},
      {reinterpret_cast<void**>(&ctx->gb.rank1), C * 4},
      {reinterpret_cast<void**>(&ctx->gb.pk), C * 4},
      {reinterpret_cast<void**>(&ctx->gb.ord23), 2 * align_up(C, 64) * 4},
      {reinterpret_cast<void**>(&ctx->gb.rank2), C * 4},
      {reinterpret_cast<void**>(&ctx->gb.c4), C * 16},
      {reinterpret_cast<void**>(&ctx->spec_x), size_t(kSpecMax) * align_up(C, 64) * 16},
      {reinterpret_cast<void**>(&ctx->spec_z), size_t(kSpecMax) * align_up(C, 64) * 4},
      {reinterpret_cast<void**>(&ctx->keep8), C},
      {reinterpret_cast<void**>(&ctx->y8), C * 4},
      {reinterpret_cast<void**>(&ctx->yf), C * 16},
      {reinterpret_cast<void**>(&ctx->spread), C * 4},
      {reinterpret_cast<void**>(&ctx->x0), C * 16},
      {reinterpret_cast<void**>(&ctx->x1), C * 16},
      {reinterpret_cast<void**>(&ctx->f64part), size_t(ctx->f64_blocks) * kP * 8},
      {reinterpret_cast<void**>(&ctx->scan_tmp), ((C + 1 + 1023) / 1024 + 1) * 8},
      {reinterpret_cast<void**>(&ctx->gb.cx), size_t(nx) * align_up(C, 64) * 4},
      {reinterpret_cast<void**>(&ctx->gb.node_sig), (p.variant & FGBD_VARIANT_SIGMA_PAIR) ? C * 4 : 0},
      {reinterpret_cast<void**>(&ctx->xbest), (p.variant & FGBD_VARIANT_GLOBAL_Q) ? C * 16 : 0},
      {reinterpret_cast<void**>(&ctx->w4), wide ? 0 : C * 16},
      {reinterpret_cast<void**>(&ctx->w2), wide ? 0 : C * 8},
      {reinterpret_cast<void**>(&ctx->wne.part), wide ? size_t(w_blocks) * wP * 8 : 0},
      {reinterpret_cast<void**>(&ctx->wne.tot), wide ? wP * 8 : 0},
      {reinterpret_cast<void**>(&ctx->wne.S), wide ? wD * wD * 8 : 0},
      {reinterpret_cast<void**>(&ctx->wne.V), wide ? (wD * wD + wD) * 4 : 0},
      {reinterpret_cast<void**>(&ctx->wne.lam), wide ? wD * 8 : 0},
      {reinterpret_cast<void**>(&ctx->wne.done), wide ? 4 : 0},
  };
  size_t total = 0;
  for (const Item& it : items) total = align_up(total, 256) + it.bytes;
  total = align_up(total, 256);
  if (cudaMalloc(&ctx->mem, total) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return FGBD_ENOMEM;
  }
  ctx->mem_bytes = total;
  size_t off = 0;
  for (const Item& it : items) {
    off = align_up(off, 256);
    *it.ptr = static_cast<char*>(ctx->mem) + off;
    off += it.bytes;
  }
  ctx->sb.count_stride = kMaxRadix * tiles;
  ctx->sb.keys[0] = static_cast<uint32_t*>(keys0);
  ctx->sb.keys[1] = static_cast<uint32_t*>(keys1);
  ctx->sb.vals[0] = static_cast<uint32_t*>(vals0);
  ctx->sb.vals[1] = static_cast<uint32_t*>(vals1);
  ctx->gb.nx = nx;
  ctx->gb.cx_stride = int(align_up(C, 64));
  if (!(p.variant & FGBD_VARIANT_SIGMA_PAIR)) ctx->gb.node_sig = nullptr;
  if (!(p.variant & FGBD_VARIANT_GLOBAL_Q)) ctx->xbest = nullptr;
  if (wide) {
    ctx->w4 = nullptr;
    ctx->w2 = nullptr;
  }
  if (!wide) {
    ctx->gb.cx = nullptr;
    ctx->wne = WideNe{};
  }
  ctx->wne.blocks = wide ? w_blocks : 0;
  // all of it zeroed once: every index array then holds indices inside the
  // context's buffers even before a build has written it (the kernels bound
  // every index they write by n <= capacity, so this stays true)
  bool ok = cudaMemset(ctx->mem, 0, total) == cudaSuccess;
  const unsigned long long limit = kWaitLimitNs;
  ok = ok && cudaMemcpy(&ctx->sc->wait_limit_ns, &limit, sizeof(limit), cudaMemcpyHostToDevice) == cudaSuccess;
  const uint32_t mode = (p.variant & FGBD_VARIANT_SIGMA_NODE) ? kSigmaNode
                        : (p.variant & FGBD_VARIANT_SIGMA_PAIR) ? kSigmaPair : kSigmaEdge;
  const uint32_t pooled = (p.variant & FGBD_VARIANT_POOLED_PATCH) ? 1u : 0u;
  ok = ok && cudaMemcpy(&ctx->sc->sigma_mode, &mode, sizeof(mode), cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemcpy(&ctx->sc->pooled_patch, &pooled, sizeof(pooled), cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaMemcpy(&ctx->sc->fslr_factor, &p.fslr_factor, sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
  for (cudaEvent_t* e : {&ctx->ev_fork, &ctx->ev_filter, &ctx->ev_join})
    ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
  ok = ok && cudaDeviceSynchronize() == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    release_batch_objects(ctx);
    cudaFree(ctx->mem);
    delete ctx;
    return FGBD_ECUDA;
  }
  *out = ctx;
  return FGBD_OK;
}

void fgbd_ctx_destroy(fgbd_ctx* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  for (cudaEvent_t e : ctx->ev)
    if (e) cudaEventDestroy(e);
  release_batch_objects(ctx);
  for (int i = 0; i < 2; ++i)
    for (cudaEvent_t e : {ctx->ev_in[i], ctx->ev_run[i], ctx->ev_out[i]})
      if (e) cudaEventDestroy(e);
  for (cudaStream_t st : {ctx->h2d, ctx->d2h})
    if (st) cudaStreamDestroy(st);
  cudaFree(ctx->stage);
  cudaFree(ctx->dmem);
  cudaFree(ctx->mem);
  delete ctx;
}

const char* fgbd_last_error(const fgbd_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

fgbd_status fgbd_build_graph(fgbd_ctx* ctx, const int32_t* xyz, int64_t n, void* stream) {
  NvtxRange nvtx_("fgbd_build_graph");
  if (!ctx) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  return do_build(ctx, xyz, n, as_stream(stream));
}

fgbd_status fgbd_estimate_noise(fgbd_ctx* ctx, const void* rgb, int32_t dtype, double* sigma_est,
                                double* sigma_est_host, void* stream) {
  NvtxRange nvtx_("fgbd_estimate_noise");
  if (!ctx) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  const cudaStream_t st = as_stream(stream);
  fgbd_status s = do_estimate(ctx, rgb, dtype, sigma_est, st);
  if (s != FGBD_OK || !sigma_est_host) return s;
  s = take_device_status(ctx, st);
  FGBD_CUDA(ctx, cudaMemcpy(sigma_est_host, &ctx->sc->sigma_est, sizeof(double), cudaMemcpyDeviceToHost));
  return s;
}

fgbd_status fgbd_select_filter(fgbd_ctx* ctx, const void* rgb, int32_t dtype, const double* sigma_est,
                               int32_t* q_out, int32_t* q_host, void* stream) {
  NvtxRange nvtx_("fgbd_select_filter");
  if (!ctx) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  const cudaStream_t st = as_stream(stream);
  fgbd_status s = do_select(ctx, rgb, dtype, sigma_est, q_out, nullptr, FGBD_F32, st);
  if (s != FGBD_OK || !q_host) return s;
  s = take_device_status(ctx, st);
  FGBD_CUDA(ctx, cudaMemcpy(q_host, &ctx->sc->q_sel, sizeof(int32_t), cudaMemcpyDeviceToHost));
  return s;
}

fgbd_status fgbd_denoise(fgbd_ctx* ctx, const void* rgb_in, int32_t in_dtype, int32_t q, void* rgb_out,
                         int32_t out_dtype, void* stream) {
  NvtxRange nvtx_("fgbd_denoise");
  if (!ctx) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  const cudaStream_t st = as_stream(stream);
  if (!ctx->has_graph) return FGBD_ESTATE;
  if (!dtype_ok(out_dtype)) return FGBD_EINVAL;
  if (ctx->n > 0 && !rgb_out) return FGBD_EINVAL;
  if (q < 0) {
    if (!ctx->has_sel) return FGBD_ESTATE;
    FGBD_LAUNCH(ctx, "filter_output", st,
                launch_output(filter_args(ctx, 1, 0, nullptr, rgb_out, out_dtype, ctx->noise_dtype), st));
    return FGBD_OK;
  }
  if (q > kQCap || !dtype_ok(in_dtype)) return FGBD_EINVAL;
  if (ctx->n > 0 && !rgb_in) return FGBD_EINVAL;
  if (ctx->n > 0) {
    FGBD_LAUNCH(ctx, "gather_colors", st,
                launch_gather_colors(rgb_in, in_dtype, ctx->n, ctx->gb.perm1, ctx->y8, ctx->yf, st));
  }
  // the gathered colours and filter buffers now hold this call's data
  if (rgb_in != ctx->noise_rgb || in_dtype != ctx->noise_dtype) {
    ctx->has_noise = false;
    ctx->spec_depth = 0;
    ctx->noise_rgb = nullptr;
  }
  ctx->has_sel = false;
  cudaError_t e = cudaSuccess;
  zero_region(ctx, offsetof(DevScalars, ysq_keep), offsetof(DevScalars, sel_end_), st, &e);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "memset");
  const FilterArgs a = filter_args(ctx, 1, q, nullptr, rgb_out, out_dtype, in_dtype);
  FGBD_LAUNCH(ctx, "filter_fixed", st, launch_filter(a, filter_grid_for(ctx, ctx->n), st));
  return FGBD_OK;
}

fgbd_status fgbd_run(fgbd_ctx* ctx, const int32_t* xyz, int64_t n, const void* rgb_in, int32_t in_dtype,
                     void* rgb_out, int32_t out_dtype, void* stream) {
  NvtxRange nvtx_("fgbd_run");
  if (!ctx) return FGBD_EINVAL;
  if (!dtype_ok(in_dtype) || !dtype_ok(out_dtype)) return FGBD_EINVAL;
  if (n > 0 && (!rgb_in || !rgb_out)) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  const cudaStream_t st = as_stream(stream);
  const fgbd_ctx::RunKey key{xyz, n, rgb_in, in_dtype, rgb_out, out_dtype};
  // a caller that is itself capturing this stream gets the kernels, not a graph launch
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    cap = cudaStreamCaptureStatusActive;
  }
  const bool replayable = ctx->graphs_on && !ctx->timing && n > 0 && cap == cudaStreamCaptureStatusNone;
  if (replayable) {
    for (size_t i = 0; i < ctx->run_graphs.size(); ++i) {
      if (!(ctx->run_graphs[i].key == key)) continue;
      fgbd_ctx::RunGraph rg = ctx->run_graphs[i];
      FGBD_CUDA(ctx, cudaGraphLaunch(rg.exec, st));
      ctx->run_graphs.erase(ctx->run_graphs.begin() + long(i));
      ctx->run_graphs.push_back(rg);
      mark_run_done(ctx, key, rg.launches);
      return FGBD_OK;
    }
    bool seen = false;
    for (const auto& k : ctx->run_seen) seen |= k == key;
    if (seen) return capture_run(ctx, key, st);
    ctx->run_seen.push_back(key);
    if (ctx->run_seen.size() > 16) ctx->run_seen.erase(ctx->run_seen.begin());
  }
  return direct_run(ctx, key, st);
}

fgbd_status fgbd_run_host(fgbd_ctx* ctx, const int32_t* xyz, int64_t n, const void* rgb_in, int32_t in_dtype,
                          void* rgb_out, int32_t out_dtype, void* stream) {
  NvtxRange nvtx_("fgbd_run_host");
  if (!ctx) return FGBD_EINVAL;
  if (!dtype_ok(in_dtype) || !dtype_ok(out_dtype)) return FGBD_EINVAL;
  if (n < 0 || n > ctx->capacity) return FGBD_EINVAL;
  if (n > 0 && (!xyz || !rgb_in || !rgb_out)) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  const cudaStream_t st = as_stream(stream);
  const size_t C = size_t(ctx->capacity);
  const size_t xyz_b = align_up(C * 12, 256), col_b = align_up(C * 12, 256);  // float colours are the larger
  const size_t slot_b = xyz_b + 2 * col_b;
  if (!ctx->stage) {
    // first call: the staging slots, copy streams and events (this synchronises the device once)
    if (cudaMalloc(&ctx->stage, 2 * slot_b) != cudaSuccess) {
      cudaGetLastError();
      ctx->stage = nullptr;
      return FGBD_ENOMEM;
    }
    ctx->stage_bytes = 2 * slot_b;
    FGBD_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->h2d, cudaStreamNonBlocking));
    FGBD_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->d2h, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      FGBD_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_in[i], cudaEventDisableTiming));
      FGBD_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_run[i], cudaEventDisableTiming));
      FGBD_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_out[i], cudaEventDisableTiming));
    }
  }
  const int slot = ctx->stage_next;
  ctx->stage_next ^= 1;
  // the call before the previous one used this slot: its output copy must be done
  // (so its host buffers are free again) before the slot is refilled
  if (ctx->stage_used[slot]) FGBD_CUDA(ctx, cudaEventSynchronize(ctx->ev_out[slot]));
  char* base = static_cast<char*>(ctx->stage) + size_t(slot) * slot_b;
  int32_t* dxyz = reinterpret_cast<int32_t*>(base);
  void* din = base + xyz_b;
  void* dout = base + xyz_b + col_b;
  const size_t in_b = size_t(n) * (in_dtype == FGBD_U8 ? 3 : 12);
  const size_t out_b = size_t(n) * (out_dtype == FGBD_U8 ? 3 : 12);
  // inputs on the copy stream, at once: they overlap the previous call's device work
  if (n > 0) {
    FGBD_CUDA(ctx, cudaMemcpyAsync(dxyz, xyz, size_t(n) * 12, cudaMemcpyHostToDevice, ctx->h2d));
    FGBD_CUDA(ctx, cudaMemcpyAsync(din, rgb_in, in_b, cudaMemcpyHostToDevice, ctx->h2d));
  }
  FGBD_CUDA(ctx, cudaEventRecord(ctx->ev_in[slot], ctx->h2d));
  FGBD_CUDA(ctx, cudaStreamWaitEvent(st, ctx->ev_in[slot], 0));
  ctx->stage_used[slot] = true;
  const fgbd_status s = fgbd_run(ctx, dxyz, n, din, in_dtype, dout, out_dtype, stream);
  if (s != FGBD_OK) return s;
  // the output on the other copy stream, after the run
  FGBD_CUDA(ctx, cudaEventRecord(ctx->ev_run[slot], st));
  FGBD_CUDA(ctx, cudaStreamWaitEvent(ctx->d2h, ctx->ev_run[slot], 0));
  if (n > 0) FGBD_CUDA(ctx, cudaMemcpyAsync(rgb_out, dout, out_b, cudaMemcpyDeviceToHost, ctx->d2h));
  FGBD_CUDA(ctx, cudaEventRecord(ctx->ev_out[slot], ctx->d2h));
  return FGBD_OK;
}

fgbd_status fgbd_run_reuse(fgbd_ctx* ctx, const int32_t* xyz, int64_t n, const void* rgb_in, int32_t in_dtype,
                           void* rgb_out, int32_t out_dtype, void* stream) {
  NvtxRange nvtx_("fgbd_run_reuse");
  if (!ctx) return FGBD_EINVAL;
  if (!dtype_ok(in_dtype) || !dtype_ok(out_dtype)) return FGBD_EINVAL;
  if (n > 0 && (!rgb_in || !rgb_out)) return FGBD_EINVAL;
  if (!ctx->ever_selected) return FGBD_ESTATE;
  DeviceGuard g(ctx->device);
  const cudaStream_t st = as_stream(stream);
  const fgbd_status s = do_build(ctx, xyz, n, st);
  if (s != FGBD_OK) return s;
  if (ctx->n > 0)
    FGBD_LAUNCH(ctx, "gather_colors", st,
                launch_gather_colors(rgb_in, in_dtype, ctx->n, ctx->gb.perm1, ctx->y8, ctx->yf, st));
  cudaError_t e = cudaSuccess;
  zero_region(ctx, offsetof(DevScalars, ysq_keep), offsetof(DevScalars, sel_end_), st, &e);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "memset");
  FilterArgs a = filter_args(ctx, 1, 0, nullptr, rgb_out, out_dtype, in_dtype);
  a.q_src = &ctx->sc->q_sel;
  FGBD_LAUNCH(ctx, "filter_reuse", st, launch_filter(a, filter_grid_for(ctx, ctx->n), st));
  return FGBD_OK;
}

fgbd_status fgbd_run_batch(fgbd_ctx* const* ctxs, const int32_t* const* xyz, const int64_t* n,
                           const void* const* rgb_in, const int32_t* in_dtype, void* const* rgb_out,
                           const int32_t* out_dtype, int32_t count, void* stream) {
  NvtxRange nvtx_("fgbd_run_batch");
  if (count < 0 || count > FGBD_BATCH_MAX) return FGBD_EINVAL;
  if (count == 0) return FGBD_OK;
  if (!ctxs || !xyz || !n || !rgb_in || !in_dtype || !rgb_out || !out_dtype) return FGBD_EINVAL;
  for (int f = 0; f < count; ++f) {
    fgbd_ctx* c = ctxs[f];
    if (!c || c->device != ctxs[0]->device) return FGBD_EINVAL;
    for (int h = 0; h < f; ++h)
      if (ctxs[h] == c) return FGBD_EINVAL;  // one frame per context
    if (!dtype_ok(in_dtype[f]) || !dtype_ok(out_dtype[f])) return FGBD_EINVAL;
    if (n[f] < 0 || n[f] > c->capacity) return FGBD_EINVAL;
    if (n[f] > 0 && (!xyz[f] || !rgb_in[f] || !rgb_out[f])) return FGBD_EINVAL;
  }
  DeviceGuard g(ctxs[0]->device);
  const cudaStream_t st = as_stream(stream);
  fgbd_ctx* lead = ctxs[0];
  std::vector<fgbd_ctx*> cv(ctxs, ctxs + count);
  std::vector<uint64_t> uids;
  for (int f = 0; f < count; ++f) uids.push_back(ctxs[f]->uid);
  std::vector<fgbd_ctx::RunKey> keys;
  for (int f = 0; f < count; ++f) keys.push_back({xyz[f], n[f], rgb_in[f], in_dtype[f], rgb_out[f], out_dtype[f]});
  bool timing = false;
  for (int f = 0; f < count; ++f) timing |= ctxs[f]->timing;
  const BatchShape shape = shape_for(lead->device, size_class(keys));
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    cap = cudaStreamCaptureStatusActive;
  }
  // like fgbd_run: the second call with the same contexts and arguments records a
  // CUDA graph of the whole batch, later calls launch it
  if (lead->graphs_on && !timing && cap == cudaStreamCaptureStatusNone) {
    for (size_t i = 0; i < lead->batch_graphs.size(); ++i) {
      const fgbd_ctx::BatchGraph& bg = lead->batch_graphs[i];
      if (bg.uids != uids || bg.ctxs != cv || !(bg.keys == keys)) continue;
      if (bg.shape.seg_frames != shape.seg_frames || bg.shape.scatter_threads != shape.scatter_threads ||
          bg.shape.filter_threads != shape.filter_threads || bg.shape.filter_per_sm != shape.filter_per_sm)
        continue;
      FGBD_CUDA(lead, cudaGraphLaunch(bg.exec, st));
      const bool seg = shape.seg_frames > 0 && seg_eligible(cv, keys);
      for (int f = 0; f < count; ++f) {
        mark_run_done(ctxs[f], keys[f], bg.launches[f]);
        if (seg) ctxs[f]->spec_depth = std::min(kSpecMax, int(ctxs[f]->params.q_max));
      }
      return FGBD_OK;
    }
    bool seen = false;
    for (const auto& e : lead->batch_seen) seen |= e.first == uids && e.second == keys;
    if (seen) return capture_batch(lead, cv, keys, shape, st);
    lead->batch_seen.push_back({uids, keys});
    if (lead->batch_seen.size() > 8) lead->batch_seen.erase(lead->batch_seen.begin());
  }
  return direct_batch(cv, keys, shape, st);
}

fgbd_status fgbd_get_batch_shape(int32_t device, int64_t mean_points, fgbd_batch_shape* out) {
  if (!out || mean_points < 0) return FGBD_EINVAL;
  const int cls = int(std::floor(std::log2(std::max(double(mean_points), 1.0))));
  const BatchShape b = shape_for(device, cls);
  std::memset(out, 0, sizeof(*out));
  out->seg_frames = b.seg_frames;
  out->scatter_threads = b.scatter_threads;
  out->filter_threads = b.filter_threads;
  out->filter_blocks_per_sm = b.filter_per_sm;
  return FGBD_OK;
}

fgbd_status fgbd_set_batch_shape(int32_t device, int64_t mean_points, const fgbd_batch_shape* shape) {
  if (mean_points < 0) return FGBD_EINVAL;
  const int cls = int(std::floor(std::log2(std::max(double(mean_points), 1.0))));
  if (!shape) {
    store_shape(device, cls, nullptr);
    return FGBD_OK;
  }
  BatchShape b;
  b.seg_frames = shape->seg_frames;
  b.scatter_threads = shape->scatter_threads;
  b.filter_threads = shape->filter_threads;
  b.filter_per_sm = shape->filter_blocks_per_sm;
  if (!shape_ok(b)) return FGBD_EINVAL;
  store_shape(device, cls, &b);
  return FGBD_OK;
}

fgbd_status fgbd_tune_batch(fgbd_ctx* const* ctxs, const int32_t* const* xyz, const int64_t* n,
                            const void* const* rgb_in, const int32_t* in_dtype, void* const* rgb_out,
                            const int32_t* out_dtype, int32_t count, void* stream, fgbd_batch_shape* chosen) {
  NvtxRange nvtx_("fgbd_tune_batch");
  if (count < 1 || count > FGBD_BATCH_MAX) return FGBD_EINVAL;
  if (!ctxs || !xyz || !n || !rgb_in || !in_dtype || !rgb_out || !out_dtype) return FGBD_EINVAL;
  for (int f = 0; f < count; ++f) {
    fgbd_ctx* c = ctxs[f];
    if (!c || c->device != ctxs[0]->device) return FGBD_EINVAL;
    for (int h = 0; h < f; ++h)
      if (ctxs[h] == c) return FGBD_EINVAL;
    if (!dtype_ok(in_dtype[f]) || !dtype_ok(out_dtype[f])) return FGBD_EINVAL;
    if (n[f] < 0 || n[f] > c->capacity) return FGBD_EINVAL;
    if (n[f] > 0 && (!xyz[f] || !rgb_in[f] || !rgb_out[f])) return FGBD_EINVAL;
  }
  DeviceGuard g(ctxs[0]->device);
  const cudaStream_t st = as_stream(stream);
  fgbd_ctx* lead = ctxs[0];
  std::vector<fgbd_ctx*> cv(ctxs, ctxs + count);
  std::vector<fgbd_ctx::RunKey> keys;
  for (int f = 0; f < count; ++f) keys.push_back({xyz[f], n[f], rgb_in[f], in_dtype[f], rgb_out[f], out_dtype[f]});
  const int cls = size_class(keys);
  if (chosen) std::memset(chosen, 0, sizeof(*chosen));
  if (!seg_eligible(cv, keys)) {
    // only per-frame streams apply: nothing to choose (the batch does not run)
    if (chosen) chosen->seg_frames = -1;
    return FGBD_OK;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  FGBD_CUDA(lead, cudaEventCreate(&e0));
  FGBD_CUDA(lead, cudaEventCreate(&e1));
  // the median of three timed batches (after one untimed) with a shape
  auto time_shape = [&](const BatchShape& b, float* ms) -> fgbd_status {
    fgbd_status s = direct_batch(cv, keys, b, st);
    if (s != FGBD_OK) return s;
    float t[3];
    for (int r = 0; r < 3; ++r) {
      FGBD_CUDA(lead, cudaEventRecord(e0, st));
      s = direct_batch(cv, keys, b, st);
      if (s != FGBD_OK) return s;
      FGBD_CUDA(lead, cudaEventRecord(e1, st));
      FGBD_CUDA(lead, cudaEventSynchronize(e1));
      FGBD_CUDA(lead, cudaEventElapsedTime(&t[r], e0, e1));
    }
    std::sort(t, t + 3);
    *ms = t[1];
    return FGBD_OK;
  };
  // coordinate search: how the frames run (per-frame streams, or segmented
  // launches of 16, 8, 4 or 2 frames), then - if segmented - the scatter's
  // threads per tile, then the filter's block shape and blocks per SM
  BatchShape best;
  best.seg_frames = 0;
  float best_ms = 0.f;
  fgbd_status s = time_shape(best, &best_ms);
  for (int sf : {16, 8, 4, 2}) {
    if (s != FGBD_OK || sf >= count * 2) continue;  // chunks larger than the batch repeat a candidate
    BatchShape b;
    b.seg_frames = sf;
    float ms = 0.f;
    s = time_shape(b, &ms);
    if (s == FGBD_OK && ms < best_ms) {
      best = b;
      best_ms = ms;
    }
  }
  if (s == FGBD_OK && best.seg_frames > 0) {
    for (int th : {256, 1024}) {
      if (s != FGBD_OK) break;
      BatchShape b = best;
      b.scatter_threads = th;
      float ms = 0.f;
      s = time_shape(b, &ms);
      if (s == FGBD_OK && ms < best_ms) {
        best = b;
        best_ms = ms;
      }
    }
    const BatchShape sorted_best = best;
    for (const auto& cand : {std::make_pair(512, 1), std::make_pair(256, 2), std::make_pair(256, 4)}) {
      if (s != FGBD_OK) break;
      BatchShape b = sorted_best;
      b.filter_threads = cand.first;
      b.filter_per_sm = cand.second;
      if (b.filter_per_sm > filter_seg_max_per_sm(b.filter_threads)) continue;
      float ms = 0.f;
      s = time_shape(b, &ms);
      if (s == FGBD_OK && ms < best_ms) {
        best = b;
        best_ms = ms;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != FGBD_OK) return s;
  store_shape(lead->device, cls, &best);
  if (chosen) {
    chosen->seg_frames = best.seg_frames;
    chosen->scatter_threads = best.scatter_threads;
    chosen->filter_threads = best.filter_threads;
    chosen->filter_blocks_per_sm = best.filter_per_sm;
    chosen->ms = best_ms;
  }
  return FGBD_OK;
}

fgbd_status fgbd_filter_forward(fgbd_ctx* ctx, const float* rgb_in, int32_t q, double alpha, double sigma,
                                int32_t checkpoint, float* rgb_out, void* stream) {
  NvtxRange nvtx_("fgbd_filter_forward");
  if (!ctx) return FGBD_EINVAL;
  if (ctx->params.window != 1) return FGBD_ENOTIMPL;  // the adjoint rows hold six neighbours
  if (ctx->params.variant & FGBD_VARIANT_SIGMA_PAIR) return FGBD_ENOTIMPL;  // its bandwidth is one scalar
  if (!ctx->has_graph) return FGBD_ESTATE;
  if (q < 0 || q > kQCap || checkpoint < 0) return FGBD_EINVAL;
  if (!std::isfinite(alpha) || !std::isfinite(sigma) || sigma < 0.0) return FGBD_EINVAL;
  const int n = ctx->n;
  if (n > 0 && (!rgb_in || !rgb_out)) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  const cudaStream_t st = as_stream(stream);
  const int c = std::max(1, std::min(checkpoint == 0 ? 1 : int(checkpoint), std::max(int(q), 1)));
  const int grid = diff_grid(std::max(n, 1), ctx->num_sms);
  ctx->d_valid = false;
  const fgbd_status ws = diff_workspace(ctx, n, q, c, grid);
  if (ws != FGBD_OK) return ws;
  const float a = float(alpha);
  if (n > 0) {
    FGBD_LAUNCH(ctx, "diff_rows", st, launch_diff_rows(n, ctx->params.bits, sigma, ctx->gb, ctx->sc, ctx->db,
                                                       ctx->num_sms, st));
    FGBD_LAUNCH(ctx, "diff_gather", st, launch_diff_gather(n, rgb_in, ctx->gb.perm1, ctx->d_ckpt, ctx->num_sms, st));
    const float4* cur = ctx->d_ckpt;
    for (int t = 0; t < q; ++t) {
      float4* dst = ((t + 1) % c == 0) ? ctx->d_ckpt + size_t((t + 1) / c) * size_t(n) : ctx->d_pp[(t + 1) & 1];
      FGBD_LAUNCH(ctx, "diff_step", st, launch_diff_step(n, a, ctx->db, cur, dst, ctx->num_sms, st));
      cur = dst;
    }
    FGBD_LAUNCH(ctx, "diff_scatter", st, launch_diff_scatter(n, cur, ctx->gb.perm1, rgb_out, ctx->num_sms, st));
  }
  ctx->d_q = q;
  ctx->d_c = c;
  ctx->d_n = n;
  ctx->d_grid = grid;
  ctx->d_alpha = a;
  ctx->d_sigma = sigma;
  ctx->d_gen = ctx->graph_gen;
  ctx->d_valid = true;
  return FGBD_OK;
}

fgbd_status fgbd_filter_backward(fgbd_ctx* ctx, const float* grad_out, float* grad_in, double* grad_params,
                                 void* stream) {
  NvtxRange nvtx_("fgbd_filter_backward");
  if (!ctx) return FGBD_EINVAL;
  if (!ctx->d_valid || !ctx->has_graph || ctx->d_gen != ctx->graph_gen) return FGBD_ESTATE;
  const int n = ctx->d_n;
  if (n > 0 && (!grad_out || !grad_in)) return FGBD_EINVAL;
  if (!grad_params) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  const cudaStream_t st = as_stream(stream);
  const int q = ctx->d_q, c = ctx->d_c, grid = ctx->d_grid;
  const float a = ctx->d_alpha;
  int parts = 0;
  if (n > 0) {
    FGBD_LAUNCH(ctx, "diff_gather", st, launch_diff_gather(n, grad_out, ctx->gb.perm1, ctx->d_pp[0], ctx->num_sms, st));
    int ui = 0;
    int seg_t0 = -1;  // first step of the segment held in d_seg
    for (int t = q - 1; t >= 0; --t) {
      const int t0 = (t / c) * c;
      const float4* xt;
      if (t == t0) {
        xt = ctx->d_ckpt + size_t(t0 / c) * size_t(n);
      } else {
        if (seg_t0 != t0) {
          // recompute x_{t0+1} .. x_t of this segment from its checkpoint
          const float4* cur = ctx->d_ckpt + size_t(t0 / c) * size_t(n);
          for (int s = t0; s < t; ++s) {
            float4* dst = ctx->d_seg + size_t(s - t0) * size_t(n);
            FGBD_LAUNCH(ctx, "diff_step", st, launch_diff_step(n, a, ctx->db, cur, dst, ctx->num_sms, st));
            cur = dst;
          }
          seg_t0 = t0;
        }
        xt = ctx->d_seg + size_t(t - t0 - 1) * size_t(n);
      }
      FGBD_LAUNCH(ctx, "diff_back_step", st,
                  launch_diff_back_step(n, a, ctx->d_sigma, ctx->db, xt, ctx->d_pp[ui], ctx->d_pp[ui ^ 1], ctx->sc,
                                        ctx->d_part + size_t(t) * size_t(grid) * 2, ctx->num_sms, st));
      ui ^= 1;
    }
    FGBD_LAUNCH(ctx, "diff_scatter", st, launch_diff_scatter(n, ctx->d_pp[ui], ctx->gb.perm1, grad_in, ctx->num_sms, st));
    parts = q * grid;
  }
  FGBD_LAUNCH(ctx, "diff_reduce", st, launch_diff_reduce(parts, ctx->d_part, grad_params, st));
  return FGBD_OK;
}

fgbd_status fgbd_debug_set_wait_limit(fgbd_ctx* ctx, int64_t ns) {
  if (!ctx || ns < 0) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  const unsigned long long v = ns > 0 ? (unsigned long long)ns : 0ull;
  // the context's work finishes first, so no wait in flight sees the value change
  FGBD_CUDA(ctx, cudaDeviceSynchronize());
  FGBD_CUDA(ctx, cudaMemcpy(&ctx->sc->wait_limit_ns, &v, sizeof(v), cudaMemcpyHostToDevice));
  return FGBD_OK;
}

fgbd_status fgbd_debug_moments(fgbd_ctx* ctx, int64_t* s2, int64_t* s1, int64_t* n_patches) {
  if (!ctx || !s2 || !s1 || !n_patches) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  if (!ctx->has_noise || ctx->noise_dtype != FGBD_U8) return FGBD_ESTATE;
  FGBD_CUDA(ctx, cudaDeviceSynchronize());
  const int w = ctx->params.window;
  const int D = 3 * (6 * w + 1);
  std::vector<double> t(size_t(D) * D + D + 1, 0.0);
  if (w == 1) {
    DevScalars h;
    FGBD_CUDA(ctx, cudaMemcpy(&h, ctx->sc, sizeof(h), cudaMemcpyDeviceToHost));
    for (int i = 0; i < D * D; ++i) s2[i] = h.s2[i];
    for (int i = 0; i < D; ++i) s1[i] = h.s1[i];
    *n_patches = int64_t(h.n_patches);
  } else {
    // the reduced totals (exact integers held as doubles)
    FGBD_CUDA(ctx, cudaMemcpy(t.data(), ctx->wne.tot, t.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int i = 0; i < D * D; ++i) s2[i] = int64_t(t[i]);
    for (int i = 0; i < D; ++i) s1[i] = int64_t(t[size_t(D) * D + i]);
    *n_patches = int64_t(t[size_t(D) * D + D]);
  }
  for (int r = 0; r < D; ++r)
    for (int c = 0; c < r; ++c) s2[r * D + c] = 0;
  return FGBD_OK;
}

fgbd_status fgbd_debug_div(const double* a, const double* b, double* q_newton, double* q_div, int64_t n,
                           void* stream) {
  if (n < 0 || (n > 0 && (!a || !b || !q_newton || !q_div))) return FGBD_EINVAL;
  const cudaError_t e = launch_debug_div(a, b, q_newton, q_div, n, as_stream(stream));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FGBD_ECUDA;
  }
  return FGBD_OK;
}

fgbd_status fgbd_sync(fgbd_ctx* ctx, void* stream) {
  if (!ctx) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  // the output copies of fgbd_run_host run on the context's own copy stream
  if (ctx->d2h) FGBD_CUDA(ctx, cudaStreamSynchronize(ctx->d2h));
  return take_device_status(ctx, as_stream(stream));
}

fgbd_status fgbd_get_stats(fgbd_ctx* ctx, fgbd_stats* out, void* stream) {
  if (!ctx || !out) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  const fgbd_status s = take_device_status(ctx, as_stream(stream));
  DevScalars h;
  FGBD_CUDA(ctx, cudaMemcpy(&h, ctx->sc, sizeof(h), cudaMemcpyDeviceToHost));
  std::memset(out, 0, sizeof(*out));
  out->n = ctx->n;
  out->valid = (ctx->has_graph ? 1 : 0) | (ctx->has_noise ? 2 : 0) | (ctx->has_sel ? 4 : 0);
  if (ctx->has_graph) {
    out->n_edges = int64_t(h.n_edges);
    if (h.sigma_mode == kSigmaNode)
      out->sigma_g = h.node_cnt ? double(h.node_fx) / double(1ull << kDistShift) / double(h.node_cnt) : 0.0;
    else
      out->sigma_g = h.n_edges ? double(h.dist_fx) / double(1ull << kDistShift) / double(h.n_edges) : 0.0;
  }
  if (ctx->has_noise) {
    out->n_patches = int64_t(h.n_patches);
    out->patch_dim = h.pooled_patch ? 6 * ctx->params.window + 1 : 3 * (6 * ctx->params.window + 1);
    for (int i = 0; i < out->patch_dim; ++i) out->eigenvalues[i] = h.eig[i];
    out->m = h.m;
    out->tau = h.tau;
    out->sigma_est = h.sigma_est;
  }
  out->q = h.q_sel;
  out->launches = ctx->launches;
  if (ctx->has_sel) {
    out->n_keep = int64_t(h.n_keep);
    out->n_objective = std::min(h.n_J, kQCap + 1);
    for (int i = 0; i < out->n_objective; ++i) out->objective[i] = h.J[i];
  }
  return s;
}

fgbd_status fgbd_graph_csr_copy(fgbd_ctx* ctx, int64_t* row_ptr, int32_t* col, float* w, int64_t col_capacity,
                                int64_t* nnz_host, void* stream) {
  if (!ctx || !nnz_host) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  const cudaStream_t st = as_stream(stream);
  if (!ctx->has_graph) return FGBD_ESTATE;
  const fgbd_status s = take_device_status(ctx, st);
  if (s != FGBD_OK) return s;
  unsigned long long edges = 0;
  FGBD_CUDA(ctx, cudaMemcpy(&edges, &ctx->sc->n_edges, sizeof(edges), cudaMemcpyDeviceToHost));
  *nnz_host = int64_t(2 * edges);
  if (!row_ptr) return FGBD_OK;
  if (col_capacity < *nnz_host || (*nnz_host > 0 && !col)) return FGBD_EINVAL;
  const int n = ctx->n;
  FGBD_LAUNCH(ctx, "csr_degree", st, launch_csr_degree(n, ctx->gb, row_ptr, st));
  FGBD_LAUNCH(ctx, "csr_scan", st, launch_scan_i64(row_ptr, int64_t(n) + 1, ctx->scan_tmp, st));
  FGBD_LAUNCH(ctx, "csr_fill", st,
              launch_csr_fill(n, ctx->params.bits, ctx->gb, row_ptr, col, w, col_capacity, ctx->sc, st));
  FGBD_CUDA(ctx, cudaStreamSynchronize(st));
  return FGBD_OK;
}

fgbd_status fgbd_graph_export(fgbd_ctx* ctx, fgbd_graph** out, void* stream) {
  if (!ctx || !out) return FGBD_EINVAL;
  *out = nullptr;
  DeviceGuard g(ctx->device);
  const cudaStream_t st = as_stream(stream);
  if (!ctx->has_graph) return FGBD_ESTATE;
  const fgbd_status s = take_device_status(ctx, st);
  if (s != FGBD_OK) return s;
  unsigned long long edges = 0, dist = 0;
  FGBD_CUDA(ctx, cudaMemcpy(&edges, &ctx->sc->n_edges, sizeof(edges), cudaMemcpyDeviceToHost));
  FGBD_CUDA(ctx, cudaMemcpy(&dist, &ctx->sc->dist_fx, sizeof(dist), cudaMemcpyDeviceToHost));
  fgbd_graph* gr = new (std::nothrow) fgbd_graph();
  if (!gr) return FGBD_ENOMEM;
  gr->device = ctx->device;
  gr->n = ctx->n;
  gr->nnz = int64_t(2 * edges);
  gr->sigma_g = edges ? double(dist) / double(1ull << kDistShift) / double(edges) : 0.0;
  if (ctx->params.variant & FGBD_VARIANT_SIGMA_NODE) {
    unsigned long long nfx = 0, ncnt = 0;
    FGBD_CUDA(ctx, cudaMemcpy(&nfx, &ctx->sc->node_fx, sizeof(nfx), cudaMemcpyDeviceToHost));
    FGBD_CUDA(ctx, cudaMemcpy(&ncnt, &ctx->sc->node_cnt, sizeof(ncnt), cudaMemcpyDeviceToHost));
    gr->sigma_g = ncnt ? double(nfx) / double(1ull << kDistShift) / double(ncnt) : 0.0;
  }
  const size_t rp_b = align_up(size_t(gr->n + 1) * 8, 256), col_b = align_up(size_t(gr->nnz) * 4, 256);
  if (cudaMalloc(&gr->mem, rp_b + 2 * col_b) != cudaSuccess) {
    cudaGetLastError();
    delete gr;
    return FGBD_ENOMEM;
  }
  char* base = static_cast<char*>(gr->mem);
  gr->row_ptr = reinterpret_cast<int64_t*>(base);
  gr->col = reinterpret_cast<int32_t*>(base + rp_b);
  gr->w = reinterpret_cast<float*>(base + rp_b + col_b);
  const int n = ctx->n;
  cudaError_t e = cudaSuccess;
  {
    LaunchScope s1(ctx, "csr_degree", st);
    e = launch_csr_degree(n, ctx->gb, gr->row_ptr, st);
  }
  if (e == cudaSuccess) {
    LaunchScope s2(ctx, "csr_scan", st);
    e = launch_scan_i64(gr->row_ptr, int64_t(n) + 1, ctx->scan_tmp, st);
  }
  if (e == cudaSuccess) {
    LaunchScope s3(ctx, "csr_fill", st);
    e = launch_csr_fill(n, ctx->params.bits, ctx->gb, gr->row_ptr, gr->col, gr->w, gr->nnz, ctx->sc, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(gr->mem);
    delete gr;
    return cuda_fail(ctx, e, "fgbd_graph_export");
  }
  *out = gr;
  return FGBD_OK;
}

fgbd_status fgbd_graph_csr(const fgbd_graph* g, const int64_t** row_ptr, const int32_t** col, const float** w,
                           int64_t* n_host, int64_t* nnz_host, double* sigma_g_host) {
  if (!g) return FGBD_EINVAL;
  if (row_ptr) *row_ptr = g->n > 0 ? g->row_ptr : nullptr;
  if (col) *col = g->nnz > 0 ? g->col : nullptr;
  if (w) *w = g->nnz > 0 ? g->w : nullptr;
  if (n_host) *n_host = g->n;
  if (nnz_host) *nnz_host = g->nnz;
  if (sigma_g_host) *sigma_g_host = g->sigma_g;
  return FGBD_OK;
}

void fgbd_graph_free(fgbd_graph* g) {
  if (!g) return;
  DeviceGuard dg(g->device);
  cudaFree(g->mem);  // waits for work that uses it
  delete g;
}

fgbd_status fgbd_get_orders(fgbd_ctx* ctx, int32_t* orders, void* stream) {
  if (!ctx) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  if (!ctx->has_graph) return FGBD_ESTATE;
  if (ctx->n > 0 && !orders) return FGBD_EINVAL;
  const cudaStream_t st = as_stream(stream);
  FGBD_LAUNCH(ctx, "orders_export", st, launch_orders_export(ctx->n, ord_stride(ctx), ctx->gb, orders, st));
  return FGBD_OK;
}

fgbd_status fgbd_get_fslr(fgbd_ctx* ctx, float* spread, uint8_t* keep, void* stream) {
  if (!ctx) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  if (!ctx->has_sel) return FGBD_ESTATE;
  const cudaStream_t st = as_stream(stream);
  FGBD_LAUNCH(ctx, "fslr_export", st,
              launch_spread_export(ctx->n, ctx->gb.rank1, ctx->spread, ctx->keep8, spread, keep, st));
  return FGBD_OK;
}

fgbd_status fgbd_set_timing(fgbd_ctx* ctx, int32_t enable) {
  if (!ctx) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  if (enable && !ctx->ev[0]) {
    for (cudaEvent_t& e : ctx->ev) FGBD_CUDA(ctx, cudaEventCreate(&e));
  }
  ctx->timing = enable != 0;
  ctx->n_timed = 0;
  return FGBD_OK;
}

fgbd_status fgbd_get_timings(fgbd_ctx* ctx, int32_t max, int32_t* count, char* names, float* ms) {
  if (!ctx || !count || max < 0 || (max > 0 && (!names || !ms))) return FGBD_EINVAL;
  DeviceGuard g(ctx->device);
  const int k = std::min<int>(max, ctx->n_timed);
  for (int i = 0; i < k; ++i) {
    FGBD_CUDA(ctx, cudaEventSynchronize(ctx->ev[2 * i + 1]));
    float t = 0.f;
    FGBD_CUDA(ctx, cudaEventElapsedTime(&t, ctx->ev[2 * i], ctx->ev[2 * i + 1]));
    ms[i] = t;
    std::memset(names + size_t(i) * FGBD_NAME_LEN, 0, FGBD_NAME_LEN);
    std::strncpy(names + size_t(i) * FGBD_NAME_LEN, ctx->ev_name[i], FGBD_NAME_LEN - 1);
  }
  *count = k;
  ctx->n_timed = 0;
  return FGBD_OK;
}

}  // extern "C"
