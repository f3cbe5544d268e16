// api.cu - the extern "C" boundary (include/fgs.h): argument checks, per-view parameter
// tables, workspace layout, and the launches of each stage. No device memory is allocated here.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include "fgs_internal.cuh"

namespace fgs {

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = n > 0 ? n : 1;
  }
  return cached[dev];
}

// Largest tile grid accepted per view: a view's tile count must fit 20 bits so that a
// record's tile count and a 1024-record partition's sum stay well inside 32 bits.
constexpr int64_t MAX_TILES_PER_VIEW = 1 << 20;

bool build_views(const fgs_camera *cams, int n_views, Views *vs) {
  if (cams == nullptr || n_views < 1 || n_views > FGS_MAX_VIEWS) return false;
  memset(vs, 0, sizeof(Views));
  vs->n = n_views;
  int64_t tiles = 0, pixels = 0, cells = 0;
  for (int k = 0; k < n_views; ++k) {
    const fgs_camera &c = cams[k];
    if (c.width <= 0 || c.height <= 0) return false;
    if (!(isfinite(c.fx) && isfinite(c.fy) && isfinite(c.cx) && isfinite(c.cy))) return false;
    if (c.model < FGS_CAM_EQUIDISTANT || c.model > FGS_CAM_PINHOLE) return false;
    View &V = vs->v[k];
    memcpy(V.W, c.W, sizeof V.W);
    memcpy(V.b, c.b, sizeof V.b);
    V.fx = c.fx; V.fy = c.fy; V.cx = c.cx; V.cy = c.cy;
    V.model = c.model;
    for (int i = 0; i < 3; ++i)
      V.cam_pos[i] = -(c.W[i] * c.b[0] + c.W[3 + i] * c.b[1] + c.W[6 + i] * c.b[2]);
    V.width = c.width;
    V.height = c.height;
    V.tiles_x = (c.width + TILE - 1) / TILE;
    V.tiles_y = (c.height + TILE - 1) / TILE;
    if ((int64_t)V.tiles_x * V.tiles_y > MAX_TILES_PER_VIEW) return false;
    // record rects hold 16-bit tile coordinates
    if (V.tiles_x > 65535 || V.tiles_y > 65535) return false;
    V.tile_offset = tiles;
    V.pixel_offset = pixels;
    V.cells_x = (V.tiles_x + CELL - 1) / CELL;
    V.cell_offset = cells;
    tiles += (int64_t)V.tiles_x * V.tiles_y;
    pixels += (int64_t)c.width * c.height;
    cells += (int64_t)V.cells_x * ((V.tiles_y + CELL - 1) / CELL);
  }
  vs->total_tiles = tiles;
  vs->total_pixels = pixels;
  vs->total_cells = cells;
  int bits = 0;
  while (bits < 31 && ((int64_t)1 << bits) < tiles) ++bits;
  vs->tile_bits = bits;
  return true;
}

namespace {

bool gauss_ok(const fgs_gaussians *g) {
  if (g == nullptr || g->n < 0 || g->n > 0xffffffffLL || g->sh_degree < 0 || g->sh_degree > 3)
    return false;
  if (g->n > 0 && (!g->means || !g->scales || !g->quats || !g->opacities || !g->sh)) return false;
  return true;
}

GaussPtrs to_ptrs(const fgs_gaussians *g) {
  GaussPtrs p;
  p.means = g->means; p.scales = g->scales; p.quats = g->quats;
  p.opacities = g->opacities; p.sh = g->sh; p.n = g->n; p.sh_degree = g->sh_degree;
  return p;
}

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

fgs_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FGS_OK : FGS_ERR_CUDA; }

// fgs_options -> CallOpts (NULL or zero fields: the defaults); false if a field is invalid.
bool resolve_opts(const fgs_options *o, CallOpts *c) {
  *c = CallOpts();
  if (o == nullptr) return true;
  if ((o->flags & ~(uint32_t)(FGS_OPT_INSTRUMENT | FGS_OPT_NO_WAIT)) != 0) return false;
  const int f = o->fwd_pixels_per_thread, b = o->bwd_pixels_per_thread;
  if (!(f == 0 || f == 1 || f == 2 || f == 4)) return false;
  if (!(b == 0 || b == 1 || b == 2 || b == 4 || b == 8)) return false;
  if (f) c->fwd_ppt = f;
  if (b) c->bwd_ppt = b;
  c->instrument = (o->flags & FGS_OPT_INSTRUMENT) != 0;
  if (o->wait_limit) c->wait_limit = o->wait_limit;
  if (o->flags & FGS_OPT_NO_WAIT) c->wait_limit = 0;
  if ((o->main_kernel_events[0] == nullptr) != (o->main_kernel_events[1] == nullptr)) return false;
  c->ev_before = reinterpret_cast<cudaEvent_t>(o->main_kernel_events[0]);
  c->ev_after = reinterpret_cast<cudaEvent_t>(o->main_kernel_events[1]);
  return true;
}

}  // namespace
}  // namespace fgs

using namespace fgs;

extern "C" {

fgs_status fgs_workspace_size_ex(int64_t n, const fgs_camera *cams, int n_views,
                                 int64_t capacity, uint32_t flags, size_t *bytes) {
  Views vs;
  // n is bounded before it is multiplied by the view count (at most FGS_MAX_VIEWS)
  if (bytes == nullptr || n < 0 || n > 0xffffffffLL || capacity <= 0 || capacity > 0xffffffffLL ||
      !build_views(cams, n_views, &vs))
    return FGS_ERR_INVALID_ARG;
  if ((flags & ~(uint32_t)(FGS_BIN_ELLIPSE | FGS_BIN_ONESWEEP)) != 0) return FGS_ERR_INVALID_ARG;
  *bytes = ws_layout((int64_t)n_views * n, capacity, vs.total_tiles,
                     (flags & FGS_BIN_ONESWEEP) != 0).total;
  return FGS_OK;
}

fgs_status fgs_workspace_size(int64_t n, const fgs_camera *cams, int n_views, int64_t capacity,
                              size_t *bytes) {
  return fgs_workspace_size_ex(n, cams, n_views, capacity, 0u, bytes);
}

int64_t fgs_total_tiles(const fgs_camera *cams, int n_views) {
  Views vs;
  if (!build_views(cams, n_views, &vs)) return -1;
  return vs.total_tiles;
}

int64_t fgs_total_pixels(const fgs_camera *cams, int n_views) {
  Views vs;
  if (!build_views(cams, n_views, &vs)) return -1;
  return vs.total_pixels;
}

fgs_status fgs_preprocess(const fgs_gaussians *g, const fgs_camera *cams, int n_views,
                          fgs_record *records, uint32_t *tiles_touched, fgs_stream stream) {
  Views vs;
  if (!gauss_ok(g) || !build_views(cams, n_views, &vs)) return FGS_ERR_INVALID_ARG;
  if ((int64_t)n_views * g->n > 0xffffffffLL) return FGS_ERR_INVALID_ARG;
  if (g->n > 0 && (!records || !tiles_touched || !aligned(records, 16))) return FGS_ERR_INVALID_ARG;
  return cuda_status(launch_preprocess_fwd(to_ptrs(g), vs, records, tiles_touched,
                                           reinterpret_cast<cudaStream_t>(stream)));
}

fgs_status fgs_bin_sort_ex(const fgs_record *records, const uint32_t *tiles_touched, int64_t n,
                           const fgs_camera *cams, int n_views, uint64_t *keys, uint32_t *vals,
                           int64_t capacity, uint32_t *tile_ranges, int64_t *n_intersections,
                           void *workspace, size_t workspace_bytes, uint32_t flags,
                           const fgs_options *opt, fgs_stream stream) {
  Views vs;
  CallOpts co;
  if (n < 0 || n > 0xffffffffLL || capacity <= 0 || capacity > 0xffffffffLL ||
      !build_views(cams, n_views, &vs) || !resolve_opts(opt, &co))
    return FGS_ERR_INVALID_ARG;
  if ((flags & ~(uint32_t)(FGS_BIN_ELLIPSE | FGS_BIN_ONESWEEP)) != 0) return FGS_ERR_INVALID_ARG;
  // the onesweep sort bins by the rect only
  if ((flags & FGS_BIN_ELLIPSE) && (flags & FGS_BIN_ONESWEEP)) return FGS_ERR_INVALID_ARG;
  const bool onesweep = (flags & FGS_BIN_ONESWEEP) != 0;
  if ((int64_t)n_views * n > 0xffffffffLL) return FGS_ERR_INVALID_ARG;
  if (!keys || !vals || !tile_ranges || !n_intersections || !workspace) return FGS_ERR_INVALID_ARG;
  if (n > 0 && (!records || !tiles_touched || !aligned(records, 16))) return FGS_ERR_INVALID_ARG;
  if (!aligned(workspace, 256)) return FGS_ERR_INVALID_ARG;
  const WsLayout L = ws_layout((int64_t)n_views * n, capacity, vs.total_tiles, onesweep);
  if (workspace_bytes < L.total) return FGS_ERR_INVALID_ARG;
  if (onesweep)
    return cuda_status(launch_bin_sort_onesweep(records, tiles_touched, n, vs, keys, vals,
                                                capacity, tile_ranges, n_intersections,
                                                reinterpret_cast<char *>(workspace), L, co,
                                                reinterpret_cast<cudaStream_t>(stream)));
  return cuda_status(launch_bin_sort(records, tiles_touched, n, vs, keys, vals, capacity,
                                     tile_ranges, n_intersections,
                                     reinterpret_cast<char *>(workspace), L, flags, co,
                                     reinterpret_cast<cudaStream_t>(stream)));
}

fgs_status fgs_bin_sort(const fgs_record *records, const uint32_t *tiles_touched, int64_t n,
                        const fgs_camera *cams, int n_views, uint64_t *keys, uint32_t *vals,
                        int64_t capacity, uint32_t *tile_ranges, int64_t *n_intersections,
                        void *workspace, size_t workspace_bytes, fgs_stream stream) {
  return fgs_bin_sort_ex(records, tiles_touched, n, cams, n_views, keys, vals, capacity,
                         tile_ranges, n_intersections, workspace, workspace_bytes, 0u, nullptr,
                         stream);
}

fgs_status fgs_rasterize_ex(const fgs_record *records, const uint32_t *vals,
                            const uint32_t *tile_ranges, const fgs_camera *cams, int n_views,
                            const float *bg, float *images, float *final_T,
                            uint32_t *n_processed, void *workspace, size_t workspace_bytes,
                            const fgs_options *opt, fgs_stream stream) {
  Views vs;
  CallOpts co;
  if (!build_views(cams, n_views, &vs) || !resolve_opts(opt, &co)) return FGS_ERR_INVALID_ARG;
  if (!records || !vals || !tile_ranges || !images || !final_T || !n_processed || !workspace)
    return FGS_ERR_INVALID_ARG;
  if (!aligned(records, 16) || !aligned(workspace, 256) || workspace_bytes < sizeof(WsHeader))
    return FGS_ERR_INVALID_ARG;
  const float b0 = bg ? bg[0] : 0.f, b1 = bg ? bg[1] : 0.f, b2 = bg ? bg[2] : 0.f;
  WsLayout L;
  memset(&L, 0, sizeof L);
  return cuda_status(launch_raster_fwd(records, vals, tile_ranges, vs, b0, b1, b2, images,
                                       final_T, n_processed, reinterpret_cast<char *>(workspace),
                                       L, co, reinterpret_cast<cudaStream_t>(stream)));
}

fgs_status fgs_rasterize(const fgs_record *records, const uint32_t *vals,
                         const uint32_t *tile_ranges, const fgs_camera *cams, int n_views,
                         const float *bg, float *images, float *final_T, uint32_t *n_processed,
                         void *workspace, size_t workspace_bytes, fgs_stream stream) {
  return fgs_rasterize_ex(records, vals, tile_ranges, cams, n_views, bg, images, final_T,
                          n_processed, workspace, workspace_bytes, nullptr, stream);
}

fgs_status fgs_backward_raster_ex(const fgs_record *records, const uint32_t *vals,
                                  const uint32_t *tile_ranges, int64_t n, const fgs_camera *cams,
                                  int n_views, const float *bg, const float *final_T,
                                  const uint32_t *n_processed, const float *dL_dimages,
                                  void *workspace, size_t workspace_bytes,
                                  const fgs_options *opt, fgs_stream stream) {
  Views vs;
  CallOpts co;
  if (n < 0 || n > 0xffffffffLL || !build_views(cams, n_views, &vs) || !resolve_opts(opt, &co))
    return FGS_ERR_INVALID_ARG;
  const int64_t R = (int64_t)n_views * n;
  if (R > 0xffffffffLL) return FGS_ERR_INVALID_ARG;
  if (!vals || !tile_ranges || !final_T || !n_processed || !dL_dimages || !workspace)
    return FGS_ERR_INVALID_ARG;
  if (R > 0 && (!records || !aligned(records, 16))) return FGS_ERR_INVALID_ARG;
  if (!aligned(workspace, 256)) return FGS_ERR_INVALID_ARG;
  // the header, the look-back arrays, the screen-space gradient region and the tile order
  // precede every capacity-dependent region
  const WsLayout L = ws_layout(R, 1, vs.total_tiles);
  if (workspace_bytes < L.vis_rec) return FGS_ERR_INVALID_ARG;
  const float b0 = bg ? bg[0] : 0.f, b1 = bg ? bg[1] : 0.f, b2 = bg ? bg[2] : 0.f;
  return cuda_status(launch_raster_bwd(records, vals, tile_ranges, vs, b0, b1, b2, final_T,
                                       n_processed, dL_dimages, R,
                                       reinterpret_cast<char *>(workspace), L, co,
                                       reinterpret_cast<cudaStream_t>(stream)));
}

fgs_status fgs_backward_raster(const fgs_record *records, const uint32_t *vals,
                               const uint32_t *tile_ranges, int64_t n, const fgs_camera *cams,
                               int n_views, const float *bg, const float *final_T,
                               const uint32_t *n_processed, const float *dL_dimages,
                               void *workspace, size_t workspace_bytes, fgs_stream stream) {
  return fgs_backward_raster_ex(records, vals, tile_ranges, n, cams, n_views, bg, final_T,
                                n_processed, dL_dimages, workspace, workspace_bytes, nullptr,
                                stream);
}

fgs_status fgs_backward_preprocess(const fgs_gaussians *g, const fgs_camera *cams, int n_views,
                                   const fgs_record *records, const uint32_t *tiles_touched,
                                   float *d_means, float *d_scales, float *d_quats,
                                   float *d_opacities, float *d_sh, void *workspace,
                                   size_t workspace_bytes, fgs_stream stream) {
  Views vs;
  if (!gauss_ok(g) || !build_views(cams, n_views, &vs)) return FGS_ERR_INVALID_ARG;
  const int64_t R = (int64_t)n_views * g->n;
  if (R > 0xffffffffLL || !workspace || !aligned(workspace, 256)) return FGS_ERR_INVALID_ARG;
  if (g->n > 0 && (!records || !tiles_touched || !d_means || !d_scales || !d_quats ||
                   !d_opacities || !d_sh || !aligned(records, 16)))
    return FGS_ERR_INVALID_ARG;
  const WsLayout L = ws_layout(R, 1, vs.total_tiles);
  if (workspace_bytes < L.vis_rec) return FGS_ERR_INVALID_ARG;
  char *ws = reinterpret_cast<char *>(workspace);
  WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
  return cuda_status(launch_preprocess_bwd(to_ptrs(g), vs, records, tiles_touched,
                                           reinterpret_cast<const float *>(ws + L.g2d), d_means,
                                           d_scales, d_quats, d_opacities, d_sh, &hdr->status,
                                           reinterpret_cast<cudaStream_t>(stream)));
}

fgs_status fgs_backward_ex(const fgs_gaussians *g, const fgs_camera *cams, int n_views,
                           const fgs_record *records, const uint32_t *tiles_touched,
                           const uint32_t *vals, const uint32_t *tile_ranges, const float *bg,
                           const float *final_T, const uint32_t *n_processed,
                           const float *dL_dimages, float *d_means, float *d_scales,
                           float *d_quats, float *d_opacities, float *d_sh, void *workspace,
                           size_t workspace_bytes, const fgs_options *opt, fgs_stream stream) {
  if (!gauss_ok(g)) return FGS_ERR_INVALID_ARG;
  // validate both halves before launching either
  Views vs;
  CallOpts co;
  if (!build_views(cams, n_views, &vs) || !resolve_opts(opt, &co)) return FGS_ERR_INVALID_ARG;
  if (g->n > 0 && (!records || !tiles_touched || !d_means || !d_scales || !d_quats ||
                   !d_opacities || !d_sh))
    return FGS_ERR_INVALID_ARG;
  fgs_status s = fgs_backward_raster_ex(records, vals, tile_ranges, g->n, cams, n_views, bg,
                                        final_T, n_processed, dL_dimages, workspace,
                                        workspace_bytes, opt, stream);
  if (s != FGS_OK) return s;
  return fgs_backward_preprocess(g, cams, n_views, records, tiles_touched, d_means, d_scales,
                                 d_quats, d_opacities, d_sh, workspace, workspace_bytes, stream);
}

fgs_status fgs_backward(const fgs_gaussians *g, const fgs_camera *cams, int n_views,
                        const fgs_record *records, const uint32_t *tiles_touched,
                        const uint32_t *vals, const uint32_t *tile_ranges, const float *bg,
                        const float *final_T, const uint32_t *n_processed,
                        const float *dL_dimages, float *d_means, float *d_scales,
                        float *d_quats, float *d_opacities, float *d_sh, void *workspace,
                        size_t workspace_bytes, fgs_stream stream) {
  return fgs_backward_ex(g, cams, n_views, records, tiles_touched, vals, tile_ranges, bg,
                         final_T, n_processed, dL_dimages, d_means, d_scales, d_quats,
                         d_opacities, d_sh, workspace, workspace_bytes, nullptr, stream);
}

fgs_status fgs_read_status(const void *workspace, fgs_stream stream, int *status) {
  if (!workspace || !status) return FGS_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return FGS_ERR_CUDA;
  uint32_t v = 0;
  if (cudaMemcpy(&v, workspace, sizeof v, cudaMemcpyDeviceToHost) != cudaSuccess)
    return FGS_ERR_CUDA;
  *status = (int)v;
  return FGS_OK;
}

fgs_status fgs_read_counters(const void *workspace, fgs_stream stream, uint64_t *counters) {
  if (!workspace || !counters) return FGS_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return FGS_ERR_CUDA;
  if (cudaMemcpy(counters, reinterpret_cast<const char *>(workspace) + offsetof(WsHeader, counters),
                 6 * sizeof(uint64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return FGS_ERR_CUDA;
  return FGS_OK;
}

const char *fgs_status_string(int status) {
  switch (status) {
    case FGS_OK: return "ok";
    case FGS_ERR_INVALID_ARG: return "invalid argument";
    case FGS_ERR_CAPACITY: return "more intersections than the key capacity";
    case FGS_ERR_TIMEOUT: return "a bounded device-side wait gave up";
    case FGS_ERR_CUDA: return "CUDA error";
    case FGS_ERR_BOUNDS: return "an index read from memory was out of range (checked build)";
    default: return "unknown status";
  }
}

}  // extern "C"
