// noalloc.cu - fgs_bin_sort_noalloc: the tile binning + key sort of fgs_bin_sort for callers
// that cannot allocate device memory.
//
// Some callers have no way to hand this library a workspace: a plugin running inside a host
// application that owns the whole GPU memory budget and forbids allocation, or a hard real-time
// loop that must never call cudaMalloc / cudaFree (both can synchronise the device). For them,
// this entry point keeps all of the sort's scratch (status word, scan look-backs, compacted
// record list, tile-class lists, bucketed pair words) in one file-scope device array of fixed
// size, so the only memory the caller provides is the inputs and outputs.
//
// The array is part of the module: every GPU that loads the library holds it (about 12 MB)
// until the process exits. It supports at most NOALLOC_MAX_RECORDS records (views x Gaussians),
// NOALLOC_MAX_CAPACITY key slots and NOALLOC_MAX_TILES tiles over all views; larger requests
// are rejected before anything is launched.
// All calls share the one array, so calls whose work overlaps on the GPU (concurrent streams,
// threads) race; calls on one stream, one after another, are safe. Each call clears every part
// of the array that must start at zero, so the previous call's leftovers do not matter.
// The first call on a device looks up the array's device address there (once per device, with
// that device current); that first call should come before any stream capture.
#include <mutex>

#include "fgs_internal.cuh"

namespace fgs {
namespace {

constexpr int64_t NOALLOC_MAX_RECORDS = 1 << 19;
constexpr int64_t NOALLOC_MAX_CAPACITY = 1 << 19;
constexpr int64_t NOALLOC_MAX_TILES = 1 << 17;

constexpr size_t NOALLOC_BYTES =
    ws_layout_ex(NOALLOC_MAX_RECORDS, NOALLOC_MAX_CAPACITY, NOALLOC_MAX_TILES, false).total;

// The scratch itself. In host code `g_noalloc_scratch` is only a host-side stand-in for the
// symbol, never a device address: the device address is looked up per device below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
char *g_scratch_ptr[MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device, looked up once per device.
char *scratch_on_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
    g_scratch_ptr[dev] = static_cast<char *>(p);
  }
  return g_scratch_ptr[dev];
}

}  // namespace
}  // namespace fgs

using namespace fgs;

extern "C" fgs_status fgs_bin_sort_noalloc(const fgs_record *records,
                                           const uint32_t *tiles_touched, int64_t n,
                                           const fgs_camera *cams, int n_views, uint64_t *keys,
                                           uint32_t *vals, int64_t capacity,
                                           uint32_t *tile_ranges, int64_t *n_intersections,
                                           uint32_t *status, fgs_stream stream) {
  if (n < 0 || n_views < 1 || n_views > FGS_MAX_VIEWS || capacity <= 0) return FGS_ERR_INVALID_ARG;
  const int64_t R = (int64_t)n_views * n;
  // sizes beyond the fixed scratch are rejected before anything touches the device
  if (R > NOALLOC_MAX_RECORDS || capacity > NOALLOC_MAX_CAPACITY) return FGS_ERR_INVALID_ARG;
  if (!keys || !vals || !tile_ranges || !n_intersections || !status) return FGS_ERR_INVALID_ARG;
  if (n > 0 && (!records || !tiles_touched || (reinterpret_cast<uintptr_t>(records) & 15)))
    return FGS_ERR_INVALID_ARG;
  Views vs;
  if (!build_views(cams, n_views, &vs) || vs.total_tiles > NOALLOC_MAX_TILES)
    return FGS_ERR_INVALID_ARG;
  const WsLayout L = ws_layout_ex(R, capacity, vs.total_tiles, false);
  if (L.total > NOALLOC_BYTES) return FGS_ERR_INVALID_ARG;
  char *ws = scratch_on_current_device();
  if (ws == nullptr) return FGS_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (launch_bin_sort(records, tiles_touched, n, vs, keys, vals, capacity, tile_ranges,
                      n_intersections, ws, L, 0u, st) != cudaSuccess)
    return FGS_ERR_CUDA;
  // hand the device status word to the caller's buffer (a device-to-device copy, no host sync)
  if (cudaMemcpyAsync(status, ws + L.header, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess)
    return FGS_ERR_CUDA;
  return FGS_OK;
}
