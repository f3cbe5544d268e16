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
// The first call on a device looks up the array's device address there (with that device
// current); that first call should come before any stream capture. The address is kept per
// device together with the unique id of the context it was looked up in, and looked up again
// when a call finds another context current (a non-primary context, or a new primary context
// after cudaDeviceReset), so a kernel never gets an address of a module that is gone.
#include <cuda.h>

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
struct ScratchEntry {
  char *ptr = nullptr;
  unsigned long long ctx_id = 0;
};
ScratchEntry g_scratch[MAX_DEVICES];

// Unique id (for the life of the process) of the calling thread's current context, through
// driver entry points resolved by the runtime (the library does not link the driver itself).
// false if there is no current context or the entry points are unavailable. Called under g_mu.
bool current_context_id(unsigned long long *id) {
  using GetCurrent = CUresult (*)(CUcontext *);
  using GetId = CUresult (*)(CUcontext, unsigned long long *);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    resolved = true;
    void *a = nullptr, *b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) ==
            cudaSuccess && qa == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) ==
            cudaSuccess && qb == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<GetCurrent>(a);
      get_id = reinterpret_cast<GetId>(b);
    }
  }
  if (get_current == nullptr || get_id == nullptr) return false;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the scratch array in the current context of the current device.
char *scratch_on_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = 0;
  const bool known = current_context_id(&id);
  ScratchEntry &e = g_scratch[dev];
  if (known && e.ptr != nullptr && e.ctx_id == id) return e.ptr;
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return nullptr;
  // the lookup makes the runtime's context current if none was: take its id now
  if (!known && !current_context_id(&id)) {
    e.ptr = nullptr;  // no id to check a later call against: look up again next time
    return static_cast<char *>(p);
  }
  e.ptr = static_cast<char *>(p);
  e.ctx_id = id;
  return e.ptr;
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
  // sizes beyond the fixed scratch are rejected before anything touches the device; n is
  // bounded before it is multiplied by the view count
  if (n < 0 || n > NOALLOC_MAX_RECORDS || n_views < 1 || n_views > FGS_MAX_VIEWS ||
      capacity <= 0 || capacity > NOALLOC_MAX_CAPACITY)
    return FGS_ERR_INVALID_ARG;
  const int64_t R = (int64_t)n_views * n;
  if (R > NOALLOC_MAX_RECORDS) return FGS_ERR_INVALID_ARG;
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
                      n_intersections, ws, L, 0u, CallOpts(), st) != cudaSuccess)
    return FGS_ERR_CUDA;
  // hand the device status word to the caller's buffer (a device-to-device copy, no host sync)
  if (cudaMemcpyAsync(status, ws + L.header, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess)
    return FGS_ERR_CUDA;
  return FGS_OK;
}
