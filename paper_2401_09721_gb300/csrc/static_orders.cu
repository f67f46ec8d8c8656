// fgbd_scan_orders_static: the scan-order radix sort without any device allocation.
//
// Some callers cannot call cudaMalloc at the moment they need the scan orders:
// a real-time frame loop where an allocation would stall the frame, plug-ins
// whose host application owns all device memory, or services on a GPU with a
// fixed memory budget.  This
// entry point runs the same histogram and radix-sort kernels as
// fgbd_build_graph, but its scratch (key/value ping-pong buffers, per-tile
// digit counts, coordinate histograms, orders, ranks) lives in one file-scope device array of
// fixed size, reserved on every GPU that loads the library until the process
// exits.  The caller passes the coordinates and the output buffer.
#include <mutex>

#include "../../include/fgbd.h"
#include "fgbd_internal.cuh"

using namespace fgbd;

namespace {

constexpr size_t kMaxPts = FGBD_STATIC_MAX_POINTS;
constexpr size_t kMaxTiles = (kMaxPts + kSortTile - 1) / kSortTile;

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// byte offsets inside the scratch array
constexpr size_t kOffScalars = 0;
constexpr size_t kOffKeys0 = align256(kOffScalars + sizeof(DevScalars));
constexpr size_t kOffKeys1 = align256(kOffKeys0 + kMaxPts * 4);
constexpr size_t kOffVals0 = align256(kOffKeys1 + kMaxPts * 4);
constexpr size_t kOffVals1 = align256(kOffVals0 + kMaxPts * 4);
constexpr size_t kOffTileCounts = align256(kOffVals1 + kMaxPts * 4);
constexpr size_t kOffPerm1 = align256(kOffTileCounts + size_t(kSlgPasses) * kMaxRadix * kMaxTiles * 4);
constexpr size_t kOffRank1 = align256(kOffPerm1 + kMaxPts * 4);
constexpr size_t kOffPk = align256(kOffRank1 + kMaxPts * 4);
constexpr size_t kOffOrd23 = align256(kOffPk + kMaxPts * 4);
constexpr size_t kOffRank2 = align256(kOffOrd23 + 2 * kMaxPts * 4);
constexpr size_t kScratchBytes = align256(kOffRank2 + kMaxPts * 4);

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" fgbd_status fgbd_scan_orders_static(const int32_t* xyz, int64_t n64, int32_t bits, int32_t* orders,
                                               uint32_t* status, void* stream) {
  if (n64 < 0 || n64 > int64_t(kMaxPts)) return FGBD_EINVAL;
  if (bits < 1 || bits > kMaxBits) return FGBD_EINVAL;
  if (n64 > 0 && (!xyz || !orders)) return FGBD_EINVAL;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned char* base = nullptr;
  if (scratch_for_current_device(&base) != cudaSuccess) {
    cudaGetLastError();
    return FGBD_ECUDA;
  }
  DevScalars* sc = reinterpret_cast<DevScalars*>(base + kOffScalars);
  // the array keeps the previous call's contents: clear the status word and
  // the coordinate histograms (the per-tile digit counts are rewritten by every pass)
  if (cudaMemsetAsync(sc, 0, sizeof(DevScalars), st) != cudaSuccess) {
    cudaGetLastError();
    return FGBD_ECUDA;
  }
  const int n = int(n64);
  if (n > 0) {
    int num_sms = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return FGBD_ECUDA;
    }
    SortBufs sb{};
    sb.keys[0] = reinterpret_cast<uint32_t*>(base + kOffKeys0);
    sb.keys[1] = reinterpret_cast<uint32_t*>(base + kOffKeys1);
    sb.vals[0] = reinterpret_cast<uint32_t*>(base + kOffVals0);
    sb.vals[1] = reinterpret_cast<uint32_t*>(base + kOffVals1);
    sb.tile_counts = reinterpret_cast<uint32_t*>(base + kOffTileCounts);
    sb.count_stride = int(size_t(kMaxRadix) * kMaxTiles);
    GraphBufs gb{};
    gb.perm1 = reinterpret_cast<int32_t*>(base + kOffPerm1);
    gb.rank1 = reinterpret_cast<int32_t*>(base + kOffRank1);
    gb.pk = reinterpret_cast<uint32_t*>(base + kOffPk);
    gb.ord23 = reinterpret_cast<int32_t*>(base + kOffOrd23);
    gb.rank2 = reinterpret_cast<int32_t*>(base + kOffRank2);
    if (launch_coord_hist(xyz, n, bits, sc, &sb, num_sms, st) != cudaSuccess) {
      cudaGetLastError();
      return FGBD_ECUDA;
    }
    // cap = n: the C2 and C3 orders lie n apart in the ord23 array
    for (int p = 0; p < kSlgPasses; ++p) {
      if (launch_sort_pass(slg_pass_args(p, xyz, n, bits, n, sb, gb, sc), st) != cudaSuccess ||
          (p == 0 && launch_slab_sort(n, bits, n, sb, gb, sc, st) != cudaSuccess)) {
        cudaGetLastError();
        return FGBD_ECUDA;
      }
    }
    // the three orders in input indices, written into the caller's [3][n] array
    if (launch_orders_export(n, n, gb, orders, st) != cudaSuccess) {
      cudaGetLastError();
      return FGBD_ECUDA;
    }
  }
  if (status && cudaMemcpyAsync(status, &sc->status, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    return FGBD_ECUDA;
  }
  return FGBD_OK;
}
